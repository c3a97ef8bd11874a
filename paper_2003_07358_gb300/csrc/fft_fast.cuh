// Column-first 2-D DFT of the zero-padded image (fast path), included by nufft.cu.
//
// Forward (F Z x): step A of the column transform reads the real image directly
// (Z fused: deapodisation, placement of pixel p at grid index p mod K) for the
// n2 grid columns that carry the image only; step B (when K1 = N1c * N2c needs
// two passes) works on those n2 columns too; the row DFT then runs over every
// grid row, reading only the n2 image columns.  Bytes per channel: 4N + 16N +
// 2 x 16N + 16N + 32N = 100N (N = n1 n2), against 132N for the row-first order.
// Adjoint: row DFT^H of every row storing only the n2 image columns, step B^H,
// then step A^H with the crop, Z^T, real part and eta fused into its store.
// Row transforms use a sequence-major shared buffer padded every 8 elements,
// which makes the Stockham stores bank-conflict-free.
// Included inside namespace fhs of nufft.cu (it uses that file's FFT building blocks).

__device__ __forceinline__ int colmap(int cc, int n2, int K2) { return cc < n2 / 2 ? cc : K2 - n2 + cc; }

template <int N>
struct Row2Cfg {
  static constexpr int S = RowCfg<N>::S;
  static constexpr int NT = RowCfg<N>::NT;
  static constexpr int SMEM = (N * S + (N * S) / 8) * 8;   // padded float2 buffer, bytes
};

// Row DFT of grid rows r0 .. r0 + S - 1 (all K1 rows over the grid).  Forward:
// only the n2 image columns are read (the others are zero); inverse: only those
// columns are stored.
template <int N>
__global__ void __launch_bounds__(Row2Cfg<N>::NT) k_row2(float2* __restrict__ grid, int K1, int n2, int inv,
                                                         const float2* __restrict__ tw, int twstride) {
  constexpr int S = Row2Cfg<N>::S, NT = Row2Cfg<N>::NT;
  extern __shared__ float2 smem[];
  const int l = blockIdx.y;
  const int r0 = blockIdx.x * S;
  float2* gl = grid + (size_t)l * K1 * N;
  const int h2 = n2 / 2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * S; idx += NT) {
    int s = idx / N, n = idx % N;
    bool in = n < h2 || n >= N - h2;
    float2 v = make_float2(0.f, 0.f);
    if ((inv || in) && r0 + s < K1) v = gl[(size_t)(r0 + s) * N + n];
    smem[pix<true>(s * N + n)] = v;
  }
  __syncthreads();
  smem_fft<N, S, NT, true, true>(smem, tw, twstride, inv != 0);
#pragma unroll
  for (int idx = threadIdx.x; idx < N * S; idx += NT) {
    int s = idx / N, n = idx % N;
    bool in = n < h2 || n >= N - h2;
    if ((inv && !in) || r0 + s >= K1) continue;
    gl[(size_t)(r0 + s) * N + n] = smem[pix<true>(s * N + n)];
  }
}

// Step A forward with Z fused: for group g, rows rho = N2c i + g (i < N = N1c) of the
// zero-padded, deapodised image, compact image columns [c0, c0 + W); DFT along i;
// twiddle exp(-2 pi i g i / K1) when the column DFT has two passes.
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::NT) k_colA_fwd(const float* __restrict__ x, float2* __restrict__ grid,
                                                            const float* __restrict__ sr, const float* __restrict__ sc,
                                                            int n1, int n2, int K1, int K2, int N2c,
                                                            const float2* __restrict__ tw, int twN, int twK) {
  constexpr int W = ColCfg<N>::W, NT = ColCfg<N>::NT;
  extern __shared__ float2 smem[];
  const int l = blockIdx.z, g = blockIdx.y, c0 = blockIdx.x * W;
  const float* xl = x + (size_t)l * n1 * n2;
  const int h1 = n1 / 2, h2 = n2 / 2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    int rho = N2c * i + g;
    int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    float val = 0.f;
    if (r >= 0 && cc < n2) {
      int c = cc < h2 ? cc + h2 : cc - h2;
      val = xl[(size_t)r * n2 + c] * sr[r] * sc[c];
    }
    smem[i * W + w] = make_float2(val, 0.f);
  }
  __syncthreads();
  smem_fft<N, W, NT>(smem, tw, twN, false);
  float2* gl = grid + (size_t)l * K1 * K2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    if (cc >= n2) continue;
    float2 v = smem[i * W + w];
    if (N2c > 1) v = cmul(v, __ldg(&tw[(size_t)(g * i) * twK]));
    gl[(size_t)(N2c * i + g) * K2 + colmap(cc, n2, K2)] = v;
  }
}

// Step B (both directions): group k1, rows N2c k1 + i (i < N = N2c), compact columns.
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::NT) k_colB(float2* __restrict__ grid, int n2, int K1, int K2, int inv,
                                                        const float2* __restrict__ tw, int twN) {
  constexpr int W = ColCfg<N>::W, NT = ColCfg<N>::NT;
  extern __shared__ float2 smem[];
  const int l = blockIdx.z, k1 = blockIdx.y, c0 = blockIdx.x * W;
  float2* gl = grid + (size_t)l * K1 * K2 + (size_t)N * k1 * K2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    smem[i * W + w] = cc < n2 ? gl[(size_t)i * K2 + colmap(cc, n2, K2)] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  smem_fft<N, W, NT>(smem, tw, twN, inv != 0);
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    if (cc < n2) gl[(size_t)i * K2 + colmap(cc, n2, K2)] = smem[i * W + w];
  }
}

// Step A^H with the crop fused: conjugate twiddle, inverse DFT along i, then for the
// rows that carry the image out[l][r][c] (+)= eta_l s_r s_c Re(.).
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::NT) k_colA_adj(const float2* __restrict__ grid, float* __restrict__ out,
                                                            const float* __restrict__ sr, const float* __restrict__ sc,
                                                            const float* __restrict__ eta, int accumulate, int n1,
                                                            int n2, int K1, int K2, int N2c,
                                                            const float2* __restrict__ tw, int twN, int twK) {
  constexpr int W = ColCfg<N>::W, NT = ColCfg<N>::NT;
  extern __shared__ float2 smem[];
  const int l = blockIdx.z, g = blockIdx.y, c0 = blockIdx.x * W;
  const float2* gl = grid + (size_t)l * K1 * K2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    float2 v = make_float2(0.f, 0.f);
    if (cc < n2) {
      v = gl[(size_t)(N2c * i + g) * K2 + colmap(cc, n2, K2)];
      if (N2c > 1) v = cmul(v, cconj(__ldg(&tw[(size_t)(g * i) * twK])));
    }
    smem[i * W + w] = v;
  }
  __syncthreads();
  smem_fft<N, W, NT>(smem, tw, twN, true);
  const float e = eta ? eta[l] : 1.f;
  const int h1 = n1 / 2, h2 = n2 / 2;
  float* ol = out + (size_t)l * n1 * n2;
#pragma unroll
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int cc = c0 + w;
    int rho = N2c * i + g;
    int r = rho < h1 ? rho + h1 : (rho >= K1 - h1 ? rho - (K1 - h1) : -1);
    if (r < 0 || cc >= n2) continue;
    int c = cc < h2 ? cc + h2 : cc - h2;
    float val = e * sr[r] * sc[c] * smem[i * W + w].x;
    size_t o = (size_t)r * n2 + c;
    ol[o] = accumulate ? ol[o] + val : val;
  }
}

#include "fft_reg.cuh"

// ------------------------------------------------------------- dispatch
template <int N, bool INV>
static void rowr_n(const Cube& cb, float2* grid, const float2* tw, int Kmax, cudaStream_t st) {
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_rowr<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegRow<N>::SMEM); attr = true; }
  dim3 grd(cb.K1, cb.L);
  k_rowr<N, INV><<<grd, RegRow<N>::NT, RegRow<N>::SMEM, st>>>(grid, cb.K1, cb.n2, tw, Kmax / N);
  note_launches(1);
}

template <int N>
static void row2_n(const Cube& cb, float2* grid, int inv, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 2048) {
    if (inv) rowr_n<N, true>(cb, grid, tw, Kmax, st);
    else rowr_n<N, false>(cb, grid, tw, Kmax, st);
    return;
  }
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_row2<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  constexpr int S = Row2Cfg<N>::S;
  dim3 grd((cb.K1 + S - 1) / S, cb.L);
  k_row2<N><<<grd, Row2Cfg<N>::NT, Row2Cfg<N>::SMEM, st>>>(grid, cb.K1, cb.n2, inv, tw, Kmax / N);
  note_launches(1);
}

template <int N>
static void colA_fwd_n(const Cube& cb, const float* x, float2* grid, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 64 && N <= 256) {
    static bool attr_r = false;
    if (!attr_r) { cudaFuncSetAttribute(k_colA_fwd_r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegCol<N>::SMEM); attr_r = true; }
    dim3 grd((cb.n2 + 31) / 32, cb.N2c, cb.L);
    k_colA_fwd_r<N><<<grd, 256, RegCol<N>::SMEM, st>>>(x, grid, cb.d_scale_r, cb.d_scale_c, cb.n1, cb.n2, cb.K1,
                                                       cb.K2, cb.N2c, tw, Kmax / N, Kmax / cb.K1);
    note_launches(1);
    return;
  }
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_colA_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  constexpr int W = ColCfg<N>::W;
  dim3 grd((cb.n2 + W - 1) / W, cb.N2c, cb.L);
  k_colA_fwd<N><<<grd, ColCfg<N>::NT, (size_t)N * W * sizeof(float2), st>>>(
      x, grid, cb.d_scale_r, cb.d_scale_c, cb.n1, cb.n2, cb.K1, cb.K2, cb.N2c, tw, Kmax / N, Kmax / cb.K1);
  note_launches(1);
}

// Step B over n2 columns of a grid with row pitch K2 (the packed transform: n2 = K2 = its
// column count, identity column map).
struct ColBDims {
  int n2, K1, K2, N1c, L;
};

static ColBDims colb_dims(const Cube& cb) { return ColBDims{cb.n2, cb.K1, cb.K2, cb.N1c, cb.L}; }

template <int N, bool INV>
static void colB_r_n(const ColBDims& d, float2* grid, const float2* tw, int Kmax, cudaStream_t st) {
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_colB_r<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegCol<N>::SMEM); attr = true; }
  dim3 grd((d.n2 + 31) / 32, d.N1c, d.L);
  k_colB_r<N, INV><<<grd, 256, RegCol<N>::SMEM, st>>>(grid, d.n2, d.K1, d.K2, tw, Kmax / N);
  note_launches(1);
}

template <int N>
static void colB_d(const ColBDims& d, float2* grid, int inv, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 64 && N <= 256) {
    if (inv) colB_r_n<N, true>(d, grid, tw, Kmax, st);
    else colB_r_n<N, false>(d, grid, tw, Kmax, st);
    return;
  }
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_colB<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  constexpr int W = ColCfg<N>::W;
  dim3 grd((d.n2 + W - 1) / W, d.N1c, d.L);
  k_colB<N><<<grd, ColCfg<N>::NT, (size_t)N * W * sizeof(float2), st>>>(grid, d.n2, d.K1, d.K2, inv, tw, Kmax / N);
  note_launches(1);
}

template <int N>
static void colB_n(const Cube& cb, float2* grid, int inv, const float2* tw, int Kmax, cudaStream_t st) {
  colB_d<N>(colb_dims(cb), grid, inv, tw, Kmax, st);
}

template <int N>
static void colA_adj_n(const Cube& cb, const float2* grid, float* out, const float* eta, bool acc, const float2* tw,
                       int Kmax, cudaStream_t st) {
  if constexpr (N >= 64 && N <= 256) {
    static bool attr_r = false;
    if (!attr_r) { cudaFuncSetAttribute(k_colA_adj_r<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegCol<N>::SMEM); attr_r = true; }
    dim3 grd((cb.n2 + 31) / 32, cb.N2c, cb.L);
    k_colA_adj_r<N><<<grd, 256, RegCol<N>::SMEM, st>>>(grid, out, cb.d_scale_r, cb.d_scale_c, eta, acc ? 1 : 0, cb.n1,
                                                       cb.n2, cb.K1, cb.K2, cb.N2c, tw, Kmax / N, Kmax / cb.K1);
    note_launches(1);
    return;
  }
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_colA_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  constexpr int W = ColCfg<N>::W;
  dim3 grd((cb.n2 + W - 1) / W, cb.N2c, cb.L);
  k_colA_adj<N><<<grd, ColCfg<N>::NT, (size_t)N * W * sizeof(float2), st>>>(
      grid, out, cb.d_scale_r, cb.d_scale_c, eta, acc ? 1 : 0, cb.n1, cb.n2, cb.K1, cb.K2, cb.N2c, tw, Kmax / N,
      Kmax / cb.K1);
  note_launches(1);
}

// Two-for-one transforms (K2 >= 2048, register row DFT).  Forward: step A packs two image
// columns per complex column into the packed scratch, step B runs on its n2/2 columns, and
// k_rowr_fwd_p unpacks each frequency pair (k, K1 - k) into two grid rows.  Adjoint:
// k_rowr_adj_p transforms each pair of grid rows and packs the Hermitian parts of two
// image columns per complex column, step B^H runs on n2/2 columns, and k_colA_adj_p
// writes the real and imaginary parts of each output as two image columns.  Bytes per
// channel and direction: 68N against 100N for the unpacked column-first order.
bool fft_forward_packed(const Cube& cb) {
  return cb.pow2 && cb.K2 >= 2048 && cb.K2 <= 8192 && cb.N1c >= 64 && cb.N1c <= 256 && cb.n2 % 64 == 0 &&
         cb.n2 * 2 == cb.K2;
}

template <int N>
static void colA_fwd_p_n(const Cube& cb, const float* x, float2* P, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 64 && N <= 256) {
    static bool attr = false;
    if (!attr) { cudaFuncSetAttribute(k_colA_fwd_p<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegCol<N>::SMEM); attr = true; }
    dim3 grd((cb.n2 / 2 + 31) / 32, cb.N2c, cb.L);
    k_colA_fwd_p<N><<<grd, 256, RegCol<N>::SMEM, st>>>(x, P, cb.d_scale_r, cb.d_scale_c, cb.n1, cb.n2, cb.K1, cb.N2c,
                                                       tw, Kmax / N, Kmax / cb.K1);
    note_launches(1);
  }
}

template <int N>
static void colB_p_n(const Cube& cb, float2* P, const float2* tw, int Kmax, cudaStream_t st) {
  // step B over the n2/2 packed columns: row pitch n2/2, identity column map
  colB_d<N>(ColBDims{cb.n2 / 2, cb.K1, cb.n2 / 2, cb.N1c, cb.L}, P, 0, tw, Kmax, st);
}

template <int N>
static void rowr_p_n(const Cube& cb, float2* grid, const float2* P, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 2048) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_rowr_fwd_p<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegRow<N>::SMEM);
      attr = true;
    }
    RowPack pk;
    pk.P = P;
    pk.N1c = cb.N1c;
    pk.lg1 = __builtin_ctz(cb.N1c);
    pk.lg2 = __builtin_ctz(cb.N2c);
    dim3 grd(cb.K1 / 2 + 1, cb.L);
    k_rowr_fwd_p<N><<<grd, RegRow<N>::NT, RegRow<N>::SMEM, st>>>(grid, cb.K1, tw, Kmax / N, pk);
    note_launches(1);
  }
}

void launch_fft_forward_fast(fhs_ctx* ctx, const Cube& cb, const float* x, float2* grid, cudaStream_t st) {
  if (fft_forward_packed(cb) && ctx->s.pack) {
    FHS_COL_SWITCH(cb.N1c, colA_fwd_p_n, cb, x, ctx->s.pack, ctx->d_tw, ctx->Kmax, st);
    if (cb.N2c > 1) { FHS_COL_SWITCH(cb.N2c, colB_p_n, cb, ctx->s.pack, ctx->d_tw, ctx->Kmax, st); }
    FHS_POW2_SWITCH(cb.K2, rowr_p_n, cb, grid, ctx->s.pack, ctx->d_tw, ctx->Kmax, st);
    return;
  }
  FHS_COL_SWITCH(cb.N1c, colA_fwd_n, cb, x, grid, ctx->d_tw, ctx->Kmax, st);
  if (cb.N2c > 1) { FHS_COL_SWITCH(cb.N2c, colB_n, cb, grid, 0, ctx->d_tw, ctx->Kmax, st); }
  FHS_POW2_SWITCH(cb.K2, row2_n, cb, grid, 0, ctx->d_tw, ctx->Kmax, st);
}

template <int N>
static void rowr_adj_p_n(const Cube& cb, const float2* grid, float2* P, const float2* tw, int Kmax, cudaStream_t st) {
  if constexpr (N >= 2048) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_rowr_adj_p<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegRowAdjP<N>::SMEM);
      attr = true;
    }
    RowPack pk;
    pk.P = P;
    pk.N1c = cb.N1c;
    pk.lg1 = __builtin_ctz(cb.N1c);
    pk.lg2 = __builtin_ctz(cb.N2c);
    dim3 grd(cb.K1 / 2 + 1, cb.L);
    k_rowr_adj_p<N><<<grd, RegRow<N>::NT, RegRowAdjP<N>::SMEM, st>>>(grid, P, cb.K1, tw, Kmax / N, pk);
    note_launches(1);
  }
}

template <int N>
static void colB_pi_n(const Cube& cb, float2* P, const float2* tw, int Kmax, cudaStream_t st) {
  colB_d<N>(ColBDims{cb.n2 / 2, cb.K1, cb.n2 / 2, cb.N1c, cb.L}, P, 1, tw, Kmax, st);
}

template <int N>
static void colA_adj_p_n(const Cube& cb, const float2* P, float* out, const float* eta, bool acc, const float2* tw,
                         int Kmax, cudaStream_t st) {
  if constexpr (N >= 64 && N <= 256) {
    static bool attr = false;
    if (!attr) { cudaFuncSetAttribute(k_colA_adj_p<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, RegCol<N>::SMEM); attr = true; }
    dim3 grd((cb.n2 / 2 + 31) / 32, cb.N2c, cb.L);
    k_colA_adj_p<N><<<grd, 256, RegCol<N>::SMEM, st>>>(P, out, cb.d_scale_r, cb.d_scale_c, eta, acc ? 1 : 0, cb.n1,
                                                       cb.n2, cb.K1, cb.N2c, tw, Kmax / N, Kmax / cb.K1);
    note_launches(1);
  }
}

void launch_fft_adjoint_fast(fhs_ctx* ctx, const Cube& cb, float2* grid, float* out, const float* eta,
                             bool accumulate, cudaStream_t st) {
  if (fft_forward_packed(cb) && ctx->s.pack && cb.n2 * 2 == cb.K2) {
    FHS_POW2_SWITCH(cb.K2, rowr_adj_p_n, cb, grid, ctx->s.pack, ctx->d_tw, ctx->Kmax, st);
    if (cb.N2c > 1) { FHS_COL_SWITCH(cb.N2c, colB_pi_n, cb, ctx->s.pack, ctx->d_tw, ctx->Kmax, st); }
    FHS_COL_SWITCH(cb.N1c, colA_adj_p_n, cb, ctx->s.pack, out, eta, accumulate, ctx->d_tw, ctx->Kmax, st);
    return;
  }
  FHS_POW2_SWITCH(cb.K2, row2_n, cb, grid, 1, ctx->d_tw, ctx->Kmax, st);
  if (cb.N2c > 1) { FHS_COL_SWITCH(cb.N2c, colB_n, cb, grid, 1, ctx->d_tw, ctx->Kmax, st); }
  FHS_COL_SWITCH(cb.N1c, colA_adj_n, cb, grid, out, eta, accumulate, ctx->d_tw, ctx->Kmax, st);
}
