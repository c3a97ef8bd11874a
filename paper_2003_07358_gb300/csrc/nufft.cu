// Measurement operator Phi = G F Z (Eq. 1) and its adjoint on GB300:
//  * Z + row DFT fused: one CTA transforms S grid rows held in shared memory
//    (Stockham autosort, radix 8/4/2, twiddles from an exp(-2 pi i k / Kmax) table);
//  * column DFT over 2n1 rows as one pass (2n1 <= 1024) or two passes of the
//    four-step factorisation K1 = N1c * N2c; the second pass leaves the rows
//    in digit-reversed order (frequency k1 + N1c k2 at row N2c k1 + k2),
//    which the interpolation kernels index directly, so no transpose pass;
//  * zero rows of the padded image are never read (pruned first column pass),
//    and the adjoint stores only the rows that survive the crop;
//  * G: one thread per visibility gathers the 7x7 Kaiser-Bessel taps; weights
//    from per-tap degree-9 polynomials fitted at context creation;
//  * G^T: one CTA per 64x64 grid tile accumulates in shared memory the
//    visibilities whose footprint touches the tile (its own sorted bin plus the
//    crossing classes of its 3 upper/left neighbours) and writes every grid
//    cell exactly once: no global atomics;
//  * l2-ball data duals (Table 2 row 4) fused into the degridder; block norms
//    in FP64 with a fixed-order two-stage reduction.
#include <cuda_runtime.h>
#include <math.h>

#include "fhs_internal.h"

namespace fhs {
// Device status word: bits set by bounded waits that gave up (read by the host).
__device__ unsigned int g_dev_status = 0;
__device__ long long g_wait_first = 0;   // first phase of the bounded waits (0: default)
}  // namespace fhs

#include "tma.cuh"

namespace fhs {

__constant__ KbPoly c_kb;

cudaError_t upload_kb_poly(const KbPoly& p) { return cudaMemcpyToSymbol(c_kb, &p, sizeof(p)); }

// ------------------------------------------------------------------ complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// ----------------------------------------------------------- R-point DFTs
// Forward sign exp(-2 pi i / R); `inv` flips the sign (unnormalised).
__device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3, bool inv) {
  float2 a0 = cadd(x0, x2), a1 = csub(x0, x2), a2 = cadd(x1, x3), a3 = csub(x1, x3);
  // -i * a3 = (a3.y, -a3.x)
  float2 mia3 = inv ? make_float2(-a3.y, a3.x) : make_float2(a3.y, -a3.x);
  x0 = cadd(a0, a2);
  x2 = csub(a0, a2);
  x1 = cadd(a1, mia3);
  x3 = csub(a1, mia3);
}

__device__ __forceinline__ void dft8(float2* v, bool inv) {
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4(e0, e1, e2, e3, inv);
  dft4(o0, o1, o2, o3, inv);
  const float c = 0.70710678118654752440f;
  float sg = inv ? 1.f : -1.f;
  // w^1 = (c, sg c), w^2 = (0, sg), w^3 = (-c, sg c)
  float2 t1 = cmul(o1, make_float2(c, sg * c));
  float2 t2 = cmul(o2, make_float2(0.f, sg));
  float2 t3 = cmul(o3, make_float2(-c, sg * c));
  v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1); v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2); v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3); v[7] = csub(e3, t3);
}

template <int R>
__device__ __forceinline__ void dftR(float2* v, bool inv) {
  if constexpr (R == 2) dft2(v[0], v[1]);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3], inv);
  else dft8(v, inv);
}

// One Stockham autosort pass over S interleaved sequences of length N held in
// shared memory as buf[n * S + s].  NT threads, each owning (N/R)*S/NT butterflies.
// PAD: one float2 of padding after every 8 elements (single-sequence buffers),
// which makes the stride-R stores of the first passes bank-conflict-free.
template <bool PAD>
__device__ __forceinline__ int pix(int e) { return PAD ? e + (e >> 3) : e; }

// SEQ: sequence-major layout buf[s * N + n] with butterflies enumerated j-fastest
// (used for row transforms); otherwise interleaved buf[n * S + s], s-fastest
// (column transforms: S = W adjacent grid columns).
template <int N, int S, int NT, int R, bool PAD = false, bool SEQ = false>
__device__ __forceinline__ void stockham_pass(float2* buf, int Ns, const float2* __restrict__ tw,
                                              int twstride, bool inv) {
  constexpr int NB = (N / R) * S;
  constexpr int PER = NB / NT;
  static_assert(PER >= 1 && PER * NT == NB, "thread count must divide the butterflies");
  float2 v[PER][R];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    int item = threadIdx.x + p * NT;
    int s = SEQ ? item / (N / R) : item % S;
    int j = SEQ ? item % (N / R) : item / S;
    int k = j % Ns;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int n = j + r * (N / R);
      v[p][r] = buf[pix<PAD>(SEQ ? s * N + n : n * S + s)];
    }
    if (Ns > 1) {
      // twiddles w^r, w = exp(-2 pi i k / (Ns R)): two table loads (w, w^4 or w^2),
      // the other powers by at most two complex products
      int step = (N / (Ns * R)) * twstride;
      float2 w1 = __ldg(&tw[k * step]);
      if (inv) w1 = cconj(w1);
      if constexpr (R == 2) {
        v[p][1] = cmul(v[p][1], w1);
      } else if constexpr (R == 4) {
        float2 w2 = __ldg(&tw[2 * k * step]);
        if (inv) w2 = cconj(w2);
        v[p][1] = cmul(v[p][1], w1);
        v[p][2] = cmul(v[p][2], w2);
        v[p][3] = cmul(v[p][3], cmul(w1, w2));
      } else {
        float2 w4 = __ldg(&tw[4 * k * step]);
        if (inv) w4 = cconj(w4);
        float2 w2 = cmul(w1, w1), w3 = cmul(w1, w2);
        v[p][1] = cmul(v[p][1], w1);
        v[p][2] = cmul(v[p][2], w2);
        v[p][3] = cmul(v[p][3], w3);
        v[p][4] = cmul(v[p][4], w4);
        v[p][5] = cmul(v[p][5], cmul(w4, w1));
        v[p][6] = cmul(v[p][6], cmul(w4, w2));
        v[p][7] = cmul(v[p][7], cmul(w4, w3));
      }
    }
    dftR<R>(v[p], inv);
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    int item = threadIdx.x + p * NT;
    int s = SEQ ? item / (N / R) : item % S;
    int j = SEQ ? item % (N / R) : item / S;
    int k = j % Ns;
    int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) {
      int n = base + r * Ns;
      buf[pix<PAD>(SEQ ? s * N + n : n * S + s)] = v[p][r];
    }
  }
  __syncthreads();
}

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// In-place DFT of S interleaved length-N sequences in shared memory.
// twstride = Kmax / N (table holds exp(-2 pi i k / Kmax)).
template <int N, int S, int NT, bool PAD = false, bool SEQ = false>
__device__ __forceinline__ void smem_fft(float2* buf, const float2* __restrict__ tw, int twstride, bool inv) {
  constexpr int LOG = ilog2c(N);
  int Ns = 1;
#pragma unroll 1
  for (int p = 0; p < LOG / 3; ++p) {
    stockham_pass<N, S, NT, 8, PAD, SEQ>(buf, Ns, tw, twstride, inv);
    Ns *= 8;
  }
  if constexpr (LOG % 3 == 2) stockham_pass<N, S, NT, 4, PAD, SEQ>(buf, Ns, tw, twstride, inv);
  if constexpr (LOG % 3 == 1) stockham_pass<N, S, NT, 2, PAD, SEQ>(buf, Ns, tw, twstride, inv);
}

// sequences per CTA for row transforms and columns per CTA for column transforms
template <int N> struct RowCfg { static constexpr int S = N >= 2048 ? 1 : 2048 / N; static constexpr int NT = N * S / 16; };
template <int N> struct ColCfg { static constexpr int W = N <= 512 ? 32 : 16; static constexpr int NT = N * W / 16; };

// Physical row of frequency row k when the column DFT used two passes.

// ------------------------------------------------------------ row kernels
// Z then row DFT: pixel rows r0..r0+S-1 of channel blockIdx.y -> grid rows (r - n1/2) mod K1.
template <int N>
__global__ void __launch_bounds__(RowCfg<N>::NT) k_row_fwd(const float* __restrict__ x, float2* __restrict__ grid,
                                                           const float* __restrict__ sr, const float* __restrict__ sc,
                                                           const float2* __restrict__ tw, int twstride, int n1, int n2,
                                                           int K1) {
  constexpr int S = RowCfg<N>::S, NT = RowCfg<N>::NT;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  const int l = blockIdx.y;
  const int r0 = blockIdx.x * S;
  const float* xl = x + (size_t)l * n1 * n2;
  const int h2 = n2 / 2;
  for (int idx = threadIdx.x; idx < N * S; idx += NT) {
    int s = idx / N, n = idx % N;
    int r = r0 + s;
    int c = n < h2 ? n + h2 : (n >= N - h2 ? n - (N - h2) : -1);
    float val = 0.f;
    if (c >= 0 && r < n1) val = xl[(size_t)r * n2 + c] * sr[r] * sc[c];
    buf[n * S + s] = make_float2(val, 0.f);
  }
  __syncthreads();
  smem_fft<N, S, NT>(buf, tw, twstride, false);
  for (int idx = threadIdx.x; idx < N * S; idx += NT) {
    int s = idx / N, n = idx % N;
    int r = r0 + s;
    if (r >= n1) continue;
    int g = (r - n1 / 2 + K1) % K1;
    grid[((size_t)l * K1 + g) * N + n] = buf[n * S + s];
  }
}

// Inverse row DFT of the grid rows that survive the crop, then crop, Z^T, real part:
// out[l][r][c] (+)= eta_l * s_r * s_c * Re(...)
template <int N>
__global__ void __launch_bounds__(RowCfg<N>::NT) k_row_adj(const float2* __restrict__ grid, float* __restrict__ out,
                                                           const float* __restrict__ sr, const float* __restrict__ sc,
                                                           const float* __restrict__ eta, int accumulate,
                                                           const float2* __restrict__ tw, int twstride, int n1, int n2,
                                                           int K1) {
  constexpr int S = RowCfg<N>::S, NT = RowCfg<N>::NT;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  const int l = blockIdx.y;
  const int r0 = blockIdx.x * S;
  for (int idx = threadIdx.x; idx < N * S; idx += NT) {
    int s = idx / N, n = idx % N;
    int r = r0 + s;
    float2 v = make_float2(0.f, 0.f);
    if (r < n1) {
      int g = (r - n1 / 2 + K1) % K1;
      v = grid[((size_t)l * K1 + g) * N + n];
    }
    buf[n * S + s] = v;
  }
  __syncthreads();
  smem_fft<N, S, NT>(buf, tw, twstride, true);
  const float e = eta ? eta[l] : 1.f;
  const int h2 = n2 / 2;
  float* ol = out + (size_t)l * n1 * n2;
  for (int idx = threadIdx.x; idx < n2 * S; idx += NT) {
    int s = idx / n2, c = idx % n2;
    int r = r0 + s;
    if (r >= n1) continue;
    int n = (c - h2 + N) % N;
    float val = e * sr[r] * sc[c] * buf[n * S + s].x;
    size_t o = (size_t)r * n2 + c;
    ol[o] = accumulate ? ol[o] + val : val;
  }
}

// -------------------------------------------------------- column kernel
// One pass of the column DFT: for group g = blockIdx.y, loads rows
// row(i) = g * gmul + i * istride (i < N), columns [c0, c0 + W), transforms
// along i, optional twiddle exp(-+2 pi i g i / K1) after (forward) or before
// (inverse) the transform, and stores back to the same rows.
// prune: rows outside the non-zero band of the zero-padded image are treated as
// zero on load (forward) or not stored (inverse).
template <int N>
__global__ void __launch_bounds__(ColCfg<N>::NT) k_col(float2* __restrict__ grid, int K1, int K2, int gmul,
                                                       int istride, int twiddle, int inv, int prune, int n1,
                                                       const float2* __restrict__ tw, int twstrideN, int twstrideK) {
  constexpr int W = ColCfg<N>::W, NT = ColCfg<N>::NT;
  extern __shared__ float2 smem[];
  float2* buf = smem;
  const int l = blockIdx.z;
  const int g = blockIdx.y;
  const int c0 = blockIdx.x * W;
  float2* gl = grid + (size_t)l * K1 * K2;
  const int h1 = n1 / 2;
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int row = g * gmul + i * istride;
    bool zero = prune && !inv && (row >= h1 && row < K1 - h1);
    float2 v = zero ? make_float2(0.f, 0.f) : gl[(size_t)row * K2 + c0 + w];
    if (twiddle && inv) {
      float2 t = __ldg(&tw[(size_t)((g * i) % K1) * twstrideK]);
      v = cmul(v, cconj(t));
    }
    buf[i * W + w] = v;
  }
  __syncthreads();
  smem_fft<N, W, NT>(buf, tw, twstrideN, inv != 0);
  for (int idx = threadIdx.x; idx < N * W; idx += NT) {
    int i = idx / W, w = idx % W;
    int row = g * gmul + i * istride;
    if (prune && inv && (row >= h1 && row < K1 - h1)) continue;
    float2 v = buf[i * W + w];
    if (twiddle && !inv) {
      float2 t = __ldg(&tw[(size_t)((g * i) % K1) * twstrideK]);
      v = cmul(v, t);
    }
    gl[(size_t)row * K2 + c0 + w] = v;
  }
}

// ----------------------------------------------------------- dispatchers
template <int N>
static void row_fwd_n(const Cube& cb, const float* x, float2* grid, const float2* tw, int Kmax, cudaStream_t st) {
  constexpr int S = RowCfg<N>::S, NT = RowCfg<N>::NT;
  size_t sm = (size_t)N * S * sizeof(float2);
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_row_fwd<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  dim3 grd((cb.n1 + S - 1) / S, cb.L);
  k_row_fwd<N><<<grd, NT, sm, st>>>(x, grid, cb.d_scale_r, cb.d_scale_c, tw, Kmax / N, cb.n1, cb.n2, cb.K1);
  note_launches(1);
}

template <int N>
static void row_adj_n(const Cube& cb, const float2* grid, float* out, const float* eta, bool acc, const float2* tw,
                      int Kmax, cudaStream_t st) {
  constexpr int S = RowCfg<N>::S, NT = RowCfg<N>::NT;
  size_t sm = (size_t)N * S * sizeof(float2);
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_row_adj<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  dim3 grd((cb.n1 + S - 1) / S, cb.L);
  k_row_adj<N><<<grd, NT, sm, st>>>(grid, out, cb.d_scale_r, cb.d_scale_c, eta, acc ? 1 : 0, tw, Kmax / N, cb.n1,
                                    cb.n2, cb.K1);
  note_launches(1);
}

template <int N>
static void col_n(const Cube& cb, float2* grid, int ngroups, int gmul, int istride, int twiddle, int inv, int prune,
                  const float2* tw, int Kmax, cudaStream_t st) {
  constexpr int W = ColCfg<N>::W, NT = ColCfg<N>::NT;
  size_t sm = (size_t)N * W * sizeof(float2);
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_col<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024); attr = true; }
  dim3 grd(cb.K2 / W, ngroups, cb.L);
  k_col<N><<<grd, NT, sm, st>>>(grid, cb.K1, cb.K2, gmul, istride, twiddle, inv, prune, cb.n1, tw, Kmax / N,
                                Kmax / cb.K1);
  note_launches(1);
}

#define FHS_POW2_SWITCH(n, FN, ...)                  \
  switch (n) {                                       \
    case 32: FN<32>(__VA_ARGS__); break;             \
    case 64: FN<64>(__VA_ARGS__); break;             \
    case 128: FN<128>(__VA_ARGS__); break;           \
    case 256: FN<256>(__VA_ARGS__); break;           \
    case 512: FN<512>(__VA_ARGS__); break;           \
    case 1024: FN<1024>(__VA_ARGS__); break;         \
    case 2048: FN<2048>(__VA_ARGS__); break;         \
    case 4096: FN<4096>(__VA_ARGS__); break;         \
    case 8192: FN<8192>(__VA_ARGS__); break;         \
    default: break;                                  \
  }

#define FHS_COL_SWITCH(n, FN, ...)                   \
  switch (n) {                                       \
    case 16: FN<16>(__VA_ARGS__); break;             \
    case 32: FN<32>(__VA_ARGS__); break;             \
    case 64: FN<64>(__VA_ARGS__); break;             \
    case 128: FN<128>(__VA_ARGS__); break;           \
    case 256: FN<256>(__VA_ARGS__); break;           \
    case 512: FN<512>(__VA_ARGS__); break;           \
    case 1024: FN<1024>(__VA_ARGS__); break;         \
    default: break;                                  \
  }

// ------------------------------------------------ mixed-radix transforms
// Grid sides K = 2^a 3^b that are not powers of two (images of 3 * 2^m pixels): Stockham
// autosort passes of radix 4, 2 and 3 between two shared-memory buffers holding W
// interleaved sequences buf[n * W + w], twiddles exp(-2 pi i k / Kmax) from the
// context's table (Kmax is a multiple of every grid side).  Rows: one CTA per image
// row; columns: one CTA per W adjacent grid columns, the whole column in one pass, so
// the grid rows stay in natural order (N1c = K1, N2c = 1).
__device__ __forceinline__ void dft3(float2& x0, float2& x1, float2& x2, bool inv) {
  const float h = 0.866025403784438646764f;                  // sqrt(3) / 2
  const float2 t = cadd(x1, x2), d = csub(x1, x2);
  const float2 m = make_float2(fmaf(-0.5f, t.x, x0.x), fmaf(-0.5f, t.y, x0.y));
  const float2 ihd = make_float2(-h * d.y, h * d.x);         // i (sqrt(3) / 2) (x1 - x2)
  x0 = cadd(x0, t);
  // forward: y1 = m - i h d, y2 = m + i h d; the inverse flips the sign of i
  x1 = inv ? cadd(m, ihd) : csub(m, ihd);
  x2 = inv ? csub(m, ihd) : cadd(m, ihd);
}

template <int R>
__device__ __forceinline__ void gen_pass(const float2* __restrict__ src, float2* __restrict__ dst, int N, int W,
                                         int Ns, const float2* __restrict__ tw, int Kmax, bool inv) {
  const int nb = (N / R) * W, tstep = Kmax / (Ns * R);
  for (int item = threadIdx.x; item < nb; item += blockDim.x) {
    const int w = item % W, j = item / W, k = j % Ns;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * (N / R)) * W + w];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 t = __ldg(&tw[(size_t)(r * k) * tstep]);
        if (inv) t = cconj(t);
        v[r] = cmul(v[r], t);
      }
    }
    if constexpr (R == 2) dft2(v[0], v[1]);
    else if constexpr (R == 3) dft3(v[0], v[1], v[2], inv);
    else dft4(v[0], v[1], v[2], v[3], inv);
    const int base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(base + r * Ns) * W + w] = v[r];
  }
}

// Runs the passes of plan p on a (b is the other buffer); returns the buffer that holds
// the transform.
__device__ float2* gen_fft(float2* a, float2* b, const GenPlan& p, int W, const float2* __restrict__ tw, int Kmax,
                           bool inv) {
  int Ns = 1;
  for (int q = 0; q < p.npass; ++q) {
    const int R = p.radix[q];
    if (R == 4) gen_pass<4>(a, b, p.n, W, Ns, tw, Kmax, inv);
    else if (R == 3) gen_pass<3>(a, b, p.n, W, Ns, tw, Kmax, inv);
    else gen_pass<2>(a, b, p.n, W, Ns, tw, Kmax, inv);
    __syncthreads();
    float2* t = a;
    a = b;
    b = t;
    Ns *= R;
  }
  return a;
}

// Z then row DFT of image row blockIdx.x of channel blockIdx.y -> grid row (r - n1/2) mod K1.
__global__ void __launch_bounds__(256) k_gen_row_fwd(const float* __restrict__ x, float2* __restrict__ grid,
                                                     const float* __restrict__ sr, const float* __restrict__ sc,
                                                     const GenPlan p, const float2* __restrict__ tw, int Kmax, int n1,
                                                     int n2, int K1) {
  extern __shared__ float2 gsm[];
  const int r = blockIdx.x, l = blockIdx.y, N = p.n, h2 = n2 / 2;
  const float* xr = x + ((size_t)l * n1 + r) * n2;
  const float s_r = sr[r];
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    const int c = n < h2 ? n + h2 : (n >= N - h2 ? n - (N - h2) : -1);
    gsm[n] = make_float2(c >= 0 ? xr[c] * s_r * sc[c] : 0.f, 0.f);
  }
  __syncthreads();
  const float2* res = gen_fft(gsm, gsm + N, p, 1, tw, Kmax, false);
  float2* gr = grid + ((size_t)l * K1 + (r - n1 / 2 + K1) % K1) * N;
  for (int n = threadIdx.x; n < N; n += blockDim.x) gr[n] = res[n];
}

// Inverse row DFT of the grid row of image row blockIdx.x, then crop, Z^T, real part:
// out[l][r][c] (+)= eta_l s_r s_c Re(...).
__global__ void __launch_bounds__(256) k_gen_row_adj(const float2* __restrict__ grid, float* __restrict__ out,
                                                     const float* __restrict__ sr, const float* __restrict__ sc,
                                                     const float* __restrict__ eta, int accumulate, const GenPlan p,
                                                     const float2* __restrict__ tw, int Kmax, int n1, int n2,
                                                     int K1) {
  extern __shared__ float2 gsm[];
  const int r = blockIdx.x, l = blockIdx.y, N = p.n, h2 = n2 / 2;
  const float2* gr = grid + ((size_t)l * K1 + (r - n1 / 2 + K1) % K1) * N;
  for (int n = threadIdx.x; n < N; n += blockDim.x) gsm[n] = gr[n];
  __syncthreads();
  const float2* res = gen_fft(gsm, gsm + N, p, 1, tw, Kmax, true);
  const float e = (eta ? eta[l] : 1.f) * sr[r];
  float* ol = out + ((size_t)l * n1 + r) * n2;
  for (int c = threadIdx.x; c < n2; c += blockDim.x) {
    const float val = e * sc[c] * res[(c - h2 + N) % N].x;
    ol[c] = accumulate ? ol[c] + val : val;
  }
}

// Column DFT (length K1 = p.n) of grid columns [c0, c0 + W) of channel blockIdx.y, in
// natural row order.  Forward: rows outside the zero-padded image band read as zero;
// inverse: only the rows of the band are stored (the crop keeps no others).
__global__ void __launch_bounds__(256) k_gen_col(float2* __restrict__ grid, const GenPlan p, int W, int K2, int n1,
                                                 int inv, const float2* __restrict__ tw, int Kmax) {
  extern __shared__ float2 gsm[];
  const int N = p.n, c0 = blockIdx.x * W, l = blockIdx.y, h1 = n1 / 2;
  float2* gl = grid + (size_t)l * N * K2;
  for (int idx = threadIdx.x; idx < N * W; idx += blockDim.x) {
    const int i = idx / W, w = idx - i * W;
    const bool zero = !inv && i >= h1 && i < N - h1;
    gsm[idx] = zero ? make_float2(0.f, 0.f) : gl[(size_t)i * K2 + c0 + w];
  }
  __syncthreads();
  const float2* res = gen_fft(gsm, gsm + N * W, p, W, tw, Kmax, inv != 0);
  for (int idx = threadIdx.x; idx < N * W; idx += blockDim.x) {
    const int i = idx / W, w = idx - i * W;
    if (inv && i >= h1 && i < N - h1) continue;
    gl[(size_t)i * K2 + c0 + w] = res[idx];
  }
}

static int gen_col_width(int K1) { return K1 <= 1536 ? 8 : 4; }

static void gen_smem_attrs() {
  static bool attr = false;
  if (attr) return;
  cudaFuncSetAttribute(k_gen_row_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(k_gen_row_adj, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(k_gen_col, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  attr = true;
}

static void launch_fft_forward_gen(fhs_ctx* ctx, const Cube& cb, const float* x, float2* grid, cudaStream_t st) {
  gen_smem_attrs();
  k_gen_row_fwd<<<dim3(cb.n1, cb.L), 256, 2 * (size_t)cb.K2 * sizeof(float2), st>>>(
      x, grid, cb.d_scale_r, cb.d_scale_c, cb.plan_c, ctx->d_tw, ctx->Kmax, cb.n1, cb.n2, cb.K1);
  const int W = gen_col_width(cb.K1);
  k_gen_col<<<dim3(cb.K2 / W, cb.L), 256, 2 * (size_t)cb.K1 * W * sizeof(float2), st>>>(
      grid, cb.plan_r, W, cb.K2, cb.n1, 0, ctx->d_tw, ctx->Kmax);
  note_launches(2);
}

static void launch_fft_adjoint_gen(fhs_ctx* ctx, const Cube& cb, float2* grid, float* out, const float* eta,
                                   bool accumulate, cudaStream_t st) {
  gen_smem_attrs();
  const int W = gen_col_width(cb.K1);
  k_gen_col<<<dim3(cb.K2 / W, cb.L), 256, 2 * (size_t)cb.K1 * W * sizeof(float2), st>>>(
      grid, cb.plan_r, W, cb.K2, cb.n1, 1, ctx->d_tw, ctx->Kmax);
  k_gen_row_adj<<<dim3(cb.n1, cb.L), 256, 2 * (size_t)cb.K2 * sizeof(float2), st>>>(
      grid, out, cb.d_scale_r, cb.d_scale_c, eta, accumulate ? 1 : 0, cb.plan_c, ctx->d_tw, ctx->Kmax, cb.n1, cb.n2,
      cb.K1);
  note_launches(2);
}

void launch_fft_forward(fhs_ctx* ctx, const Cube& cb, const float* x, float2* grid, cudaStream_t st) {
  if (!cb.pow2) {
    launch_fft_forward_gen(ctx, cb, x, grid, st);
    return;
  }
  if (ctx->path == FHS_PATH_FAST) {
    launch_fft_forward_fast(ctx, cb, x, grid, st);
    return;
  }
  FHS_POW2_SWITCH(cb.K2, row_fwd_n, cb, x, grid, ctx->d_tw, ctx->Kmax, st);
  // step A: groups g < N2c, rows N2c*i + g; twiddle after unless single pass
  FHS_COL_SWITCH(cb.N1c, col_n, cb, grid, cb.N2c, 1, cb.N2c, cb.N2c > 1 ? 1 : 0, 0, 1, ctx->d_tw, ctx->Kmax, st);
  if (cb.N2c > 1) {
    // step B: groups k1 < N1c, rows N2c*k1 + i
    FHS_COL_SWITCH(cb.N2c, col_n, cb, grid, cb.N1c, cb.N2c, 1, 0, 0, 0, ctx->d_tw, ctx->Kmax, st);
  }
}

void launch_fft_adjoint(fhs_ctx* ctx, const Cube& cb, float2* grid, float* out, const float* eta, bool accumulate,
                        cudaStream_t st) {
  if (!cb.pow2) {
    launch_fft_adjoint_gen(ctx, cb, grid, out, eta, accumulate, st);
    return;
  }
  if (ctx->path == FHS_PATH_FAST) {
    launch_fft_adjoint_fast(ctx, cb, grid, out, eta, accumulate, st);
    return;
  }
  if (cb.N2c > 1) {
    FHS_COL_SWITCH(cb.N2c, col_n, cb, grid, cb.N1c, cb.N2c, 1, 0, 1, 0, ctx->d_tw, ctx->Kmax, st);
  }
  FHS_COL_SWITCH(cb.N1c, col_n, cb, grid, cb.N2c, 1, cb.N2c, cb.N2c > 1 ? 1 : 0, 1, 1, ctx->d_tw, ctx->Kmax, st);
  FHS_POW2_SWITCH(cb.K2, row_adj_n, cb, grid, out, eta, accumulate, ctx->d_tw, ctx->Kmax, st);
}

#include "fft_fast.cuh"

// ------------------------------------------------------ Kaiser-Bessel taps
struct TapConst {
  float hi_r, lo_r, hi_c, lo_c;   // K / (2 pi) split into two floats, rows and columns
};

__host__ __device__ inline TapConst tap_const(int K1, int K2) {
  double cr = (double)K1 / (2.0 * 3.14159265358979323846);
  double cc = (double)K2 / (2.0 * 3.14159265358979323846);
  TapConst t;
  t.hi_r = (float)cr; t.lo_r = (float)(cr - (double)t.hi_r);
  t.hi_c = (float)cc; t.lo_c = (float)(cc - (double)t.hi_c);
  return t;
}

// First tap k0 = floor(t - 3.5) + 1 of t = omega * (hi + lo) and x = 2 f - 1, with
// f = t - k0 - 2.5 the offset entering the per-tap polynomials.
__device__ __forceinline__ int kb_first(float om, float hi, float lo, float& xx) {
  float p = __fmul_rn(om, hi);
  float e = __fadd_rn(__fmaf_rn(om, hi, -p), __fmul_rn(om, lo));
  float fl = floorf(__fadd_rn(p, -3.5f));
  int k0 = (int)fl + 1;
  float f = __fadd_rn(__fadd_rn(__fadd_rn(p, -(float)k0), -2.5f), e);
  xx = 2.f * f - 1.f;
  return k0;
}

// Weight of tap j (j warp-uniform for constant-cache broadcast).
__device__ __forceinline__ float kb_tap(int j, float xx) {
  float acc = c_kb.c[j][kPolyDeg];
#pragma unroll
  for (int d = kPolyDeg - 1; d >= 0; --d) acc = fmaf(acc, xx, c_kb.c[j][d]);
  return acc;
}

// First tap k0 = floor(t - 3.5) + 1 and the 7 weights phi(t - k0 - j), t = omega * (hi + lo).
// k0 depends only on p = fl(omega * hi) so that host and device agree exactly.
__device__ __forceinline__ int kb_weights(float om, float hi, float lo, float* w) {
  float p = __fmul_rn(om, hi);
  float e = __fadd_rn(__fmaf_rn(om, hi, -p), __fmul_rn(om, lo));
  float fl = floorf(__fadd_rn(p, -3.5f));
  int k0 = (int)fl + 1;
  float f = __fadd_rn(__fadd_rn(__fadd_rn(p, -(float)k0), -2.5f), e);
  float xx = 2.f * f - 1.f;
#pragma unroll
  for (int j = 0; j < kTaps; ++j) {
    float acc = c_kb.c[j][kPolyDeg];
#pragma unroll
    for (int d = kPolyDeg - 1; d >= 0; --d) acc = fmaf(acc, xx, c_kb.c[j][d]);
    w[j] = acc;
  }
  return k0;
}

// --------------------------------------------------------- degridding G
struct VisGeom {
  int K1, K2, N1c, N2c;
  int lg1, lg2;          // log2(N1c), log2(N2c) (two-pass column transforms)
  int pw;                // 1: K1 and K2 are powers of two (index wrap by masks)
  TapConst tc;
};

// Grid index k in [-K, 2K) wrapped into [0, K): a mask for power-of-two grids, one
// conditional add or subtract otherwise (K = 2^a 3^b).
__device__ __forceinline__ int wrap_k(int k, int K, int pw) {
  return pw ? (k & (K - 1)) : (k < 0 ? k + K : (k >= K ? k - K : k));
}
__device__ __forceinline__ int wrap1(int k, const VisGeom& vg) { return wrap_k(k, vg.K1, vg.pw); }
__device__ __forceinline__ int wrap2(int k, const VisGeom& vg) { return wrap_k(k, vg.K2, vg.pw); }

// Physical row of frequency row k: natural order after a one-pass column transform
// (N2c = 1), else the two-pass digit-reversed order (N1c, N2c powers of two: shifts).
__device__ __forceinline__ int phys_row2(int k, const VisGeom& vg) {
  if (vg.N2c == 1) return k;
  return ((k & (vg.N1c - 1)) << vg.lg2) | (k >> vg.lg1);
}

__device__ __forceinline__ float2 degrid_one(const float2* __restrict__ g, float2 uv, const VisGeom& vg) {
  float wc[kTaps], xr;
  int kr = kb_first(uv.y, vg.tc.hi_r, vg.tc.lo_r, xr);
  int kc = kb_weights(uv.x, vg.tc.hi_c, vg.tc.lo_c, wc);
  float2 acc = make_float2(0.f, 0.f);
  // rolled row loop (row weight evaluated per row, warp-uniform tap index) keeps the
  // register count low; the 7 loads of a row are independent
#pragma unroll 1
  for (int a = 0; a < kTaps; ++a) {
    const float wra = kb_tap(a, xr);
    int row = phys_row2(wrap1(kr + a, vg), vg);
    const float2* gr = g + (size_t)row * vg.K2;
    float2 racc = make_float2(0.f, 0.f);
#pragma unroll
    for (int b = 0; b < kTaps; ++b) {
      float2 v = __ldg(&gr[wrap2(kc + b, vg)]);
      racc.x = fmaf(wc[b], v.x, racc.x);
      racc.y = fmaf(wc[b], v.y, racc.y);
    }
    acc.x = fmaf(wra, racc.x, acc.x);
    acc.y = fmaf(wra, racc.y, acc.y);
  }
  return acc;
}

__global__ void __launch_bounds__(256) k_degrid(const float2* __restrict__ grid, const float2* __restrict__ uv,
                                                float2* __restrict__ out, const int64_t* __restrict__ vis_off,
                                                VisGeom vg) {
  const int l = blockIdx.y;
  int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vis_off[l + 1]) return;
  out[i] = degrid_one(grid + (size_t)l * vg.K1 * vg.K2, uv[i], vg);
}

// Deterministic CTA reduction of per-block sums: values v0 (||z-y||^2) and v1
// (||y - u||^2) of the visibility handled by this thread, block id b.
template <int NW>
__device__ __forceinline__ void block_partials(double v0, double v1, int b, bool valid, int B, double* sred,
                                               double* out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int b0 = __shfl_sync(0xffffffffu, valid ? b : -1, 0);
  // lanes with invalid entries contribute zero to any block
  bool uniform = __all_sync(0xffffffffu, !valid || b == b0) && b0 >= 0;
  for (int k = threadIdx.x; k < NW * 2 * B; k += blockDim.x) sred[k] = 0.0;
  __syncthreads();
  if (uniform) {
    double s0 = valid ? v0 : 0.0, s1 = valid ? v1 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      s0 += __shfl_xor_sync(0xffffffffu, s0, o);
      s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    if (lane == 0) {
      sred[(wid * 2 + 0) * B + b0] = s0;
      sred[(wid * 2 + 1) * B + b0] = s1;
    }
  } else {
    for (int bb = 0; bb < B; ++bb) {
      double s0 = (valid && b == bb) ? v0 : 0.0, s1 = (valid && b == bb) ? v1 : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (lane == 0) {
        sred[(wid * 2 + 0) * B + bb] = s0;
        sred[(wid * 2 + 1) * B + bb] = s1;
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * B; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < NW; ++w) s += sred[w * 2 * B + k];
    out[k] = s;
  }
}

// Degrid + l2-ball data dual: u = G x_hat, z = v + 2u - u_prev, d = z - y;
// per-block FP64 partial sums of ||d||^2 and ||y - u||^2; u_prev <- u.
__global__ void __launch_bounds__(256) k_degrid_pdfb(const float2* __restrict__ grid, const float2* __restrict__ uv,
                                                     const float2* __restrict__ y, const float2* __restrict__ v,
                                                     float2* __restrict__ d_out, float2* __restrict__ u_prev,
                                                     const uint8_t* __restrict__ blk,
                                                     const int64_t* __restrict__ vis_off, VisGeom vg, int B,
                                                     double* __restrict__ partials, int nparts) {
  __shared__ double sred[8 * 2 * kMaxB];
  const int l = blockIdx.y;
  int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < vis_off[l + 1];
  double v0 = 0.0, v1 = 0.0;
  int b = 0;
  if (valid) {
    float2 u = degrid_one(grid + (size_t)l * vg.K1 * vg.K2, uv[i], vg);
    float2 yy = y[i], vv = v[i], up = u_prev[i];
    float2 z = make_float2(vv.x + 2.f * u.x - up.x, vv.y + 2.f * u.y - up.y);
    float2 d = make_float2(z.x - yy.x, z.y - yy.y);
    d_out[i] = d;
    u_prev[i] = u;
    b = blk[i];
    v0 = (double)d.x * d.x + (double)d.y * d.y;
    double rx = (double)yy.x - u.x, ry = (double)yy.y - u.y;
    v1 = rx * rx + ry * ry;
  }
  block_partials<8>(v0, v1, b, valid, B, sred, partials + ((size_t)l * nparts + blockIdx.x) * 2 * B);
}

// Tile-staged degridding (fast path).  One CTA per (grid tile, channel): every
// visibility of the tile has its first tap in the tile, so its 7 x 7 footprint lies
// in the (T + 6)^2 region starting at the tile corner, which is staged in shared
// memory once (coalesced rows) and then read by all of the tile's visibilities.
// Tiles with few visibilities read the grid directly instead.  The staging is two
// TMA tensor copies (tile rows and halo rows of the digit-reversed grid, an mbarrier
// with a bounded wait) except for the last tile column, whose halo wraps around the
// grid edge and is staged with asynchronous 8-byte copies.  The staged row stride S
// (the TMA box width) is 8 mod 16 float2, so a lane's bank pair is (8 row + column) mod
// 16 of its first tap, which the host's visibility order ((8 row + column) mod 32
// distinct within 32 consecutive visibilities) makes distinct within each half-warp
// at every tap.  MODE 0 stores
// u = G x_hat; MODE 1 is the PDFB data step of k_degrid_pdfb with its per-block
// partial sums accumulated per warp in shared memory over the tile (fixed order)
// and written once per CTA: partials[l][tile][2][B].
constexpr int kDegStageMin = 96;

// acc (hi, lo) += x with an exact TwoSum of hi and x (Knuth): the pair carries the
// sum to about 2^-48 of its magnitude.
__device__ __forceinline__ void ff_accum(float2& acc, float x) {
  const float s = __fadd_rn(acc.x, x);
  const float bp = __fadd_rn(s, -acc.x);
  const float e = __fadd_rn(__fadd_rn(acc.x, -__fadd_rn(s, -bp)), __fadd_rn(x, -bp));
  acc.x = s;
  acc.y = __fadd_rn(acc.y, e);
}

// Staged row stride of the degridder (float2): the smallest S >= T + 6 with S = 8 mod 16.
__host__ __device__ inline int degrid_stage_stride(int T) { return ((T + kTaps - 1 - 8 + 15) / 16) * 16 + 8; }

template <int MODE>
__global__ void __launch_bounds__(256) k_degrid_tiled(const float2* __restrict__ grid, const float2* __restrict__ uv,
                                                      const int32_t* __restrict__ tile_off,
                                                      const int64_t* __restrict__ vis_off, VisGeom vg, int T,
                                                      int ntr, int ntc, float2* __restrict__ out,
                                                      const float2* __restrict__ y, const float2* __restrict__ v,
                                                      float2* __restrict__ u_prev, const uint8_t* __restrict__ blk,
                                                      int B, double* __restrict__ partials,
                                                      const __grid_constant__ CUtensorMap tm_rows,
                                                      const __grid_constant__ CUtensorMap tm_halo, int use_tma) {
  extern __shared__ __align__(128) float2 sg[];
  __shared__ float2 sacc[8][2][kMaxB];   // per warp, per block: float-float (hi, lo) sums
  __shared__ __align__(8) uint64_t bar;
  const int l = blockIdx.y, tau = blockIdx.x;
  const int tr = tau / ntc, tc = tau % ntc;
  const int32_t* toff = tile_off + (size_t)l * (ntr * ntc * 4 + 1);
  const int beg = toff[tau * 4], end = toff[tau * 4 + 4];
  const int64_t vbase = vis_off[l];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (MODE == 1) {
    for (int k = threadIdx.x; k < 8 * 2 * kMaxB; k += blockDim.x) (&sacc[0][0][0])[k] = make_float2(0.f, 0.f);
  }
  const float2* gl = grid + (size_t)l * vg.K1 * vg.K2;
  const int R = T + kTaps - 1, SP = degrid_stage_stride(T);
  const bool staged = end - beg >= kDegStageMin;
  const bool tma = staged && use_tma && tc + 1 < ntc;
  if (tma) {
    if (threadIdx.x == 0) {
      const int k0 = tr * T, k1 = wrap1(tr * T + T, vg);
      mbar_init(&bar, 1);
      mbar_expect_tx(&bar, (unsigned)(R * SP * sizeof(float2)));
      // view coordinates (t, r) of frequency row k: physical row r N2c + t
      const bool nat = vg.N2c == 1;
      tma_load_4d(sg, &tm_rows, tc * T, nat ? 0 : k0 >> vg.lg1, nat ? k0 : k0 & (vg.N1c - 1), l, &bar);
      tma_load_4d(sg + T * SP, &tm_halo, tc * T, nat ? 0 : k1 >> vg.lg1, nat ? k1 : k1 & (vg.N1c - 1), l, &bar);
    }
    __syncthreads();                       // the barrier is initialised before anyone waits
    mbar_wait(&bar, 0);
  } else if (staged) {
    // asynchronous 8-byte copies (all of a thread's loads in flight): lane = column,
    // warp = row
    const int lane = threadIdx.x & 31, wrp = threadIdx.x >> 5;
    for (int c0 = 0; c0 < R; c0 += 32) {
      const int cc = c0 + lane;
      if (cc >= R) continue;
      const int col = wrap2(tc * T + cc, vg);
#pragma unroll 4
      for (int rr = wrp; rr < R; rr += 8) {
        const int row = phys_row2(wrap1(tr * T + rr, vg), vg);
        const unsigned sa = (unsigned)__cvta_generic_to_shared(&sg[rr * SP + cc]);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gl + (size_t)row * vg.K2 + col));
      }
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("cp.async.wait_group 0;\n" ::);
  }
  __syncthreads();
  // the next iteration's uv is loaded one iteration ahead (its latency overlaps the taps)
  float2 w_next = beg + (int)threadIdx.x < end ? uv[vbase + beg + threadIdx.x] : make_float2(0.f, 0.f);
  for (int base = beg; base < end; base += blockDim.x) {
    const int k = base + threadIdx.x;
    const bool valid = k < end;
    const int64_t i = vbase + k;
    const float2 w = w_next;
    if (k + (int)blockDim.x < end) w_next = uv[i + blockDim.x];
    // the data-step operands are issued before the taps
    float2 yy = make_float2(0.f, 0.f), vv = yy, up = yy;
    int bk = -1;
    if (MODE == 1 && valid) {
      yy = y[i];
      vv = v[i];
      up = u_prev[i];
      bk = blk[i];
    }
    float2 u = make_float2(0.f, 0.f);
    if (valid) {
      float wc[kTaps], xr;
      const int kr = kb_first(w.y, vg.tc.hi_r, vg.tc.lo_r, xr);
      const int kc = kb_weights(w.x, vg.tc.hi_c, vg.tc.lo_c, wc);
      const int lr = wrap1(kr, vg) - tr * T, lc = wrap2(kc, vg) - tc * T;
      // the host sort puts the first tap in this tile; anything else reads the grid directly
      if (staged && lr >= 0 && lr < T && lc >= 0 && lc < T) {
        const float2* sp = sg + lr * SP + lc;
#pragma unroll 1
        for (int a = 0; a < kTaps; ++a) {
          const float wra = kb_tap(a, xr);
          float2 racc = make_float2(0.f, 0.f);
#pragma unroll
          for (int b = 0; b < kTaps; ++b) {
            const float2 g = sp[a * SP + b];
            racc.x = fmaf(wc[b], g.x, racc.x);
            racc.y = fmaf(wc[b], g.y, racc.y);
          }
          u.x = fmaf(wra, racc.x, u.x);
          u.y = fmaf(wra, racc.y, u.y);
        }
      } else {
        u = degrid_one(gl, w, vg);
      }
    }
    if (MODE == 0) {
      if (valid) out[i] = u;
      continue;
    }
    float v0 = 0.f, v1 = 0.f;
    int b = -1;
    if (valid) {
      const float2 z = make_float2(vv.x + 2.f * u.x - up.x, vv.y + 2.f * u.y - up.y);
      const float2 d = make_float2(z.x - yy.x, z.y - yy.y);
      out[i] = d;
      u_prev[i] = u;
      b = bk;
      v0 = fmaf(d.x, d.x, d.y * d.y);
      const float rx = yy.x - u.x, ry = yy.y - u.y;
      v1 = fmaf(rx, rx, ry * ry);
    }
    // valid lanes form a prefix of the CTA, so lane 0 invalid means the warp is idle
    const int b0 = __shfl_sync(0xffffffffu, b, 0);
    if (b0 < 0) continue;
    const bool uniform = __all_sync(0xffffffffu, b < 0 || b == b0);
    // FP32 tree over the 32 lanes (fixed order), then lane 0 adds the warp's sum to its
    // float-float accumulator: no FP64 arithmetic per visibility (FP64 runs at a small
    // fraction of the FP32 rate on this GPU); FP64 takes over at the CTA sum below
    for (int bb = uniform ? b0 : 0; bb < (uniform ? b0 + 1 : B); ++bb) {
      float s0 = (b == bb) ? v0 : 0.f, s1 = (b == bb) ? v1 : 0.f;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      }
      if (lane == 0) {
        ff_accum(sacc[wid][0][bb], s0);
        ff_accum(sacc[wid][1][bb], s1);
      }
    }
  }
  if (MODE == 0) return;
  __syncthreads();
  double* po = partials + ((size_t)l * ntr * ntc + tau) * 2 * B;
  for (int k = threadIdx.x; k < 2 * B; k += blockDim.x) {
    const int c = k / B, bb = k - c * B;
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += (double)sacc[w][c][bb].x + (double)sacc[w][c][bb].y;
    po[k] = s;
  }
}

// Partial sums of ||z - y||^2 per block and d = z - y (standalone l2-ball projection).
__global__ void __launch_bounds__(256) k_l2ball_partials(const float2* __restrict__ z, const float2* __restrict__ y,
                                                         float2* __restrict__ d_out, const uint8_t* __restrict__ blk,
                                                         const int64_t* __restrict__ vis_off, int B,
                                                         double* __restrict__ partials, int nparts) {
  __shared__ double sred[8 * 2 * kMaxB];
  const int l = blockIdx.y;
  int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool valid = i < vis_off[l + 1];
  double v0 = 0.0;
  int b = 0;
  if (valid) {
    float2 zz = z[i], yy = y[i];
    float2 d = make_float2(zz.x - yy.x, zz.y - yy.y);
    d_out[i] = d;
    b = blk[i];
    v0 = (double)d.x * d.x + (double)d.y * d.y;
  }
  block_partials<8>(v0, 0.0, b, valid, B, sred, partials + ((size_t)l * nparts + blockIdx.x) * 2 * B);
}

// ------------------------------------------------- preconditioned data duals
// Algorithm 2 v line with a diagonal metric U (Section 3.2), in terms of
// d = U^-1 v + Phi x_check - y (from the degridder, after v <- v / U) and w = x - y:
//   w_0 = P(d),  w_k = P(w_{k-1} - gamma U (w_{k-1} - d))  (k = 1..n_sub),  v = U (d - w),
// with P the projection onto the ball of radius eps_{l,b} centred at 0 and
// gamma = 1 / max U over the block: forward-backward sub-iterations of the U-metric
// projection.  A step stores t_k = w_{k-1} - gamma U (w_{k-1} - d) and the block partial
// sums of |t_k|^2; k_block_finalize turns them into s_k (P(t_k) = t_k (1 - s_k)), which
// the next step or the final kernel applies.
__global__ void __launch_bounds__(256) k_fb_step(const float2* __restrict__ d, float2* __restrict__ t,
                                                 const float* __restrict__ U, const float* __restrict__ gamma,
                                                 const float* __restrict__ scale_prev, const uint8_t* __restrict__ blk,
                                                 const int64_t* __restrict__ vis_off, int B, int first,
                                                 double* __restrict__ partials, int nparts) {
  __shared__ double sred[8 * 2 * kMaxB];
  const int l = blockIdx.y;
  const int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool valid = i < vis_off[l + 1];
  double v0 = 0.0;
  int b = 0;
  if (valid) {
    b = blk[i];
    const int kb = l * B + b;
    const float2 dd = d[i];
    const float keep = 1.f - scale_prev[kb];          // min(1, eps / ||.||) of the previous iterate
    const float2 src = first ? dd : t[i];
    const float2 w = make_float2(src.x * keep, src.y * keep);
    const float g = gamma[kb] * U[i];
    const float2 tn = make_float2(w.x - g * (w.x - dd.x), w.y - g * (w.y - dd.y));
    t[i] = tn;
    v0 = (double)tn.x * tn.x + (double)tn.y * tn.y;
  }
  block_partials<8>(v0, 0.0, b, valid, B, sred, partials + ((size_t)l * nparts + blockIdx.x) * 2 * B);
}

// v = U (d - P(t_n)), written over d.
__global__ void k_fb_final(float2* __restrict__ d, const float2* __restrict__ t, const float* __restrict__ U,
                           const float* __restrict__ scale, const uint8_t* __restrict__ blk,
                           const int64_t* __restrict__ vis_off, int B) {
  const int l = blockIdx.y;
  const int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vis_off[l + 1]) return;
  const float keep = 1.f - scale[l * B + blk[i]];
  const float2 tt = t[i], dd = d[i];
  const float u = U[i];
  d[i] = make_float2(u * (dd.x - tt.x * keep), u * (dd.y - tt.y * keep));
}

// v <- v * f or v <- v / f elementwise (f > 0).
__global__ void k_vis_scale(float2* __restrict__ v, const float* __restrict__ f, int64_t n, int divide) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float s = divide ? 1.f / f[i] : f[i];
  const float2 a = v[i];
  v[i] = make_float2(a.x * s, a.y * s);
}

// Per (channel, block): sum the CTA partials in order; scale = max(0, 1 - eps/||d||);
// out[2][L*B] = (||d||, ||y - u||) in FP64.
// One CTA per (channel, block): the CTA partials are summed in a fixed order
// (thread t takes p = t, t + 256, ..., then a fixed shared-memory tree), so the
// result does not depend on scheduling.  scale = max(0, 1 - eps/||d||);
// out[2][L*B] = (||d||, ||y - u||) in FP64.
__global__ void __launch_bounds__(256) k_block_finalize(const double* __restrict__ partials, int nparts, int B, int L,
                                                        const double* __restrict__ eps, float* __restrict__ scale,
                                                        double* __restrict__ out) {
  __shared__ double s0s[256], s1s[256];
  const int k = blockIdx.x;
  const int l = k / B, b = k % B;
  double s0 = 0.0, s1 = 0.0;
  for (int p = threadIdx.x; p < nparts; p += 256) {
    const double* pp = partials + ((size_t)l * nparts + p) * 2 * B;
    s0 += pp[b];
    s1 += pp[B + b];
  }
  s0s[threadIdx.x] = s0;
  s1s[threadIdx.x] = s1;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      s0s[threadIdx.x] += s0s[threadIdx.x + w];
      s1s[threadIdx.x] += s1s[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  double dn = sqrt(s0s[0]);
  double e = eps ? eps[k] : 0.0;
  // a NaN or Inf norm propagates as a NaN scale (v becomes NaN), never a silent zero
  if (scale) scale[k] = (float)(!isfinite(dn) ? nan("") : (dn > e ? 1.0 - e / dn : 0.0));
  if (out) {
    out[k] = dn;
    out[L * B + k] = sqrt(s1s[0]);
  }
}

__global__ void k_l2ball_scale(const float2* __restrict__ d, const float* __restrict__ scale,
                               const uint8_t* __restrict__ blk, const int64_t* __restrict__ vis_off, int B,
                               float2* __restrict__ v) {
  const int l = blockIdx.y;
  int64_t i = vis_off[l] + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= vis_off[l + 1]) return;
  float s = scale[l * B + blk[i]];
  float2 dd = d[i];
  v[i] = make_float2(dd.x * s, dd.y * s);
}

// ----------------------------------------------------------- gridding G^T
// One CTA per (64x64 tile, channel).  Pass (dr, dc) reads the visibilities of
// source tile (tr - dr, tc - dc) whose footprint crosses into this tile and adds
// only their taps in quadrant (dr, dc) of the source footprint, so each tap of
// each visibility lands in exactly one (tile, pass).
// Class order within a tile: 0 interior, 1 crosses down only, 2 crosses down
// and right, 3 crosses right only.
// Accumulation is in fixed point with 32-bit integer shared-memory atomics (several
// times faster than floating-point ones, and order-independent, so the result is
// bitwise deterministic), with one scale S = 2^e per tile chosen so that
// n_c |c| < 2^30 for every tap value c = w v S, with n_c the largest number of
// footprints that cover one cell of the tile (counted once per context, MODE 1) and
// |v| <= m = max over the tile's visibilities of max(|Re v|, |Im v|): no cell can
// overflow, and the resolution is n_c m / 2^30 (about 2^-23 of m for the densest
// tiles of the large workload, n_c ~ 100).

constexpr int kGridThreads = 128;                // threads per gridding CTA

// Row stride of the gridder's tile accumulators (ints): T + 8, which is 8 mod 32 for
// T = 32 or 64, so the bank of cell (r, c) is (8 r + c) mod 32 and the host's
// visibility order ((8 row + column) mod 32 of the first tap distinct within 32
// consecutive visibilities) puts the 32 lanes of a warp on 32 banks at every tap.
__host__ __device__ inline int grid_row_stride(int T) { return T + 8; }

// Source range [beg, end) of pass (dr, dc) for destination tile (tr, tc).
__device__ __forceinline__ void grid_pass_range(const int32_t* toff, int pass, int tr, int tc, int ntr, int ntc,
                                                int& sr, int& sc, int& beg, int& end) {
  const int dr = pass >> 1, dc = pass & 1;
  sr = (tr - dr + ntr) % ntr;
  sc = (tc - dc + ntc) % ntc;
  const int sidx = (sr * ntc + sc) * 4;
  if (pass == 0) { beg = toff[sidx]; end = toff[sidx + 4]; }
  else if (pass == 1) { beg = toff[sidx + 2]; end = toff[sidx + 4]; }   // crosses right: classes 2, 3
  else if (pass == 2) { beg = toff[sidx + 1]; end = toff[sidx + 3]; }   // crosses down: classes 1, 2
  else { beg = toff[sidx + 2]; end = toff[sidx + 3]; }                  // crosses both: class 2
}

__device__ __forceinline__ float pow2f(int e) { return __uint_as_float((unsigned)(e + 127) << 23); }

// Adds the 7 x 7 taps of one visibility to the tile accumulators: rows lr + a,
// columns lc + b.  ra[a] = row weight * S, wc[b] = column weight, (vx, vy) = v.
// INTERIOR: the whole footprint lies in the tile (no bounds tests); otherwise only
// rows in [a0, a1) and columns in [b0, b1) are added.  MODE 1 adds 1 per tap.
template <bool INTERIOR, int MODE>
__device__ __forceinline__ void grid_taps(int* are, int* aim, int TP, int lr, int lc, const float* ra,
                                          const float* wc, float vx, float vy, int a0, int a1, int b0, int b1) {
#pragma unroll
  for (int a = 0; a < kTaps; ++a) {
    if (!INTERIOR && (a < a0 || a >= a1)) continue;
    int* pr = are + (lr + a) * TP + lc;
    int* pi = aim + (lr + a) * TP + lc;
    const float xr = vx * ra[a], xi = vy * ra[a];
#pragma unroll
    for (int b = 0; b < kTaps; ++b) {
      if (!INTERIOR && (b < b0 || b >= b1)) continue;
      if (MODE == 1) {
        atomicAdd(pr + b, 1);
      } else {
        atomicAdd(pr + b, __float2int_rn(wc[b] * xr));
        atomicAdd(pi + b, __float2int_rn(wc[b] * xi));
      }
    }
  }
}

// MODE 0: grid the (block-scaled) values into the tile and store it; MODE 1 (once per
// context): count the footprints covering each cell and store the tile's maximum in
// ncmax[l][tile].
template <int MODE>
__global__ void __launch_bounds__(kGridThreads, 1024 / kGridThreads) k_grid(const float2* __restrict__ vals, const float* __restrict__ blk_scale,
                                              float2* __restrict__ v_write, const float2* __restrict__ uv,
                                              const uint8_t* __restrict__ blk, const int32_t* __restrict__ tile_off,
                                              const int64_t* __restrict__ vis_off, float2* __restrict__ grid,
                                              int* __restrict__ ncmax, VisGeom vg, int T, int ntr, int ntc, int B) {
  extern __shared__ __align__(16) int sacc_i[];
  constexpr int NW = kGridThreads / 32;
  __shared__ float sred[NW];
  __shared__ int sredi[NW];
  const int TP = grid_row_stride(T);     // = 8 mod 32: bank = (8 row + column) mod 32
  int* are = sacc_i;
  int* aim = are + T * TP;
  const int l = blockIdx.y;
  const int tau = blockIdx.x;
  const int tr = tau / ntc, tc = tau % ntc;
  {
    int4* z4 = reinterpret_cast<int4*>(sacc_i);
    const int n4 = (MODE == 1 ? T * TP : 2 * T * TP) / 4;
    for (int k = threadIdx.x; k < n4; k += blockDim.x) z4[k] = make_int4(0, 0, 0, 0);
  }
  const int64_t vbase = vis_off[l];
  const int32_t* toff = tile_off + (size_t)l * (ntr * ntc * 4 + 1);
  float S = 1.f;
  if (MODE == 0) {
    // ---- sweep 0: largest component magnitude over the visibilities touching the tile
    float m = 0.f;
    for (int pass = 0; pass < 4; ++pass) {
      int sr, sc, beg, end;
      grid_pass_range(toff, pass, tr, tc, ntr, ntc, sr, sc, beg, end);
      for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
        const int64_t i = vbase + k;
        const float2 val = vals[i];
        const float s = blk_scale ? blk_scale[l * B + blk[i]] : 1.f;
        m = fmaxf(m, fmaxf(fabsf(val.x * s), fabsf(val.y * s)));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.f;
#pragma unroll
    for (int w = 0; w < NW; ++w) m = fmaxf(m, sred[w]);
    const int nc = ncmax[l * ntr * ntc + tau];
    if (m > 1e-30f && nc > 0) {
      // S = 2^e <= 2^30 / (n_c m'), m' = m (1 + 2^-10) covering the roundings of v s,
      // of the row product and a kernel weight a hair above 1
      const float t = 1073741824.f / ((float)nc * (m * 1.0009765625f));
      const int e = (int)((__float_as_uint(t) >> 23) & 0xffu) - 127;   // 2^e <= t
      S = pow2f(max(-120, min(e, 120)));
    }
  } else {
    __syncthreads();
  }
  // ---- sweep 1: taps
  for (int pass = 0; pass < 4; ++pass) {
    const int dr = pass >> 1, dc = pass & 1;
    int sr, sc, beg, end;
    grid_pass_range(toff, pass, tr, tc, ntr, ntc, sr, sc, beg, end);
    // pass 0 starts with the interior class: every tap in the tile
    const int ibeg = beg, iend = pass == 0 ? toff[(sr * ntc + sc) * 4 + 1] : beg;
    for (int k = beg + threadIdx.x; k < end; k += blockDim.x) {
      const int64_t i = vbase + k;
      const float2 w = uv[i];
      float2 val = make_float2(0.f, 0.f);
      if (MODE == 0) {
        val = vals[i];
        if (blk_scale) {
          const float s = blk_scale[l * B + blk[i]];
          val.x *= s;
          val.y *= s;
        }
        if (pass == 0 && v_write) v_write[i] = val;
      }
      float wc[kTaps], ra[kTaps];
      const int kr = kb_weights(w.y, vg.tc.hi_r, vg.tc.lo_r, ra);
      const int kc = kb_weights(w.x, vg.tc.hi_c, vg.tc.lo_c, wc);
#pragma unroll
      for (int a = 0; a < kTaps; ++a) ra[a] *= S;
      // footprint start in the source tile, relative to this tile
      const int lr = wrap1(kr, vg) - sr * T - dr * T;
      const int lc = wrap2(kc, vg) - sc * T - dc * T;
      if (k >= ibeg && k < iend) {
        grid_taps<true, MODE>(are, aim, TP, lr, lc, ra, wc, val.x, val.y, 0, kTaps, 0, kTaps);
      } else {
        const int a0 = max(0, -lr), a1 = min(kTaps, T - lr);
        const int b0 = max(0, -lc), b1 = min(kTaps, T - lc);
        grid_taps<false, MODE>(are, aim, TP, lr, lc, ra, wc, val.x, val.y, a0, a1, b0, b1);
      }
    }
  }
  __syncthreads();
  if (MODE == 1) {
    int mx = 0;
    for (int q = threadIdx.x; q < T * T; q += blockDim.x) mx = max(mx, are[(q / T) * TP + q % T]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sredi[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 0; w < NW; ++w) mx = max(mx, sredi[w]);
      ncmax[l * ntr * ntc + tau] = mx;
    }
    return;
  }
  const float inv = 1.f / S;                                   // power of two: exact
  float2* gl = grid + (size_t)l * vg.K1 * vg.K2;
  for (int q = threadIdx.x; q < T * T; q += blockDim.x) {
    const int rr = q / T, cc = q % T, o = rr * TP + cc;
    const int row = phys_row2(tr * T + rr, vg);
    gl[(size_t)row * vg.K2 + tc * T + cc] = make_float2((float)are[o] * inv, (float)aim[o] * inv);
  }
}

// ------------------------------------------------------------- launchers
static VisGeom vis_geom(const Cube& cb) {
  VisGeom vg;
  vg.K1 = cb.K1; vg.K2 = cb.K2; vg.N1c = cb.N1c; vg.N2c = cb.N2c;
  vg.lg1 = __builtin_ctz(cb.N1c);
  vg.lg2 = __builtin_ctz(cb.N2c);
  vg.pw = cb.pow2 ? 1 : 0;
  vg.tc = tap_const(cb.K1, cb.K2);
  return vg;
}

int degrid_parts(const Cube& cb) { return (int)((cb.max_M + 255) / 256); }

int degrid_tiled_parts(const Cube& cb) { return cb.ntile_r * cb.ntile_c; }

static size_t degrid_tiled_smem(const Cube& cb) {
  return (size_t)(cb.tile + kTaps - 1) * degrid_stage_stride(cb.tile) * sizeof(float2);
}

// TMA descriptors for the degridder's staging (see k_degrid_tiled): the grid scratch
// of a cube viewed as a 4-D tensor of 8-byte elements, dims (K2, N2c, N1c, L) with
// row index r * N2c + t, boxes (S, 1, T, 1) and (S, 1, 6, 1).  A cube whose geometry
// does not fit (or a driver without the entry point) keeps the asynchronous copies.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

void encode_degrid_maps(fhs_ctx* ctx) {
  for (Cube& cb : ctx->cubes) encode_cube_maps(cb, ctx->s.grid, 0);
}

// Slot of cube cb's TMA maps encoded over `grid`, or -1 (asynchronous copies).
static int map_slot(const Cube& cb, const float2* grid) {
  for (int k = 0; k < kMaxLanes; ++k)
    if (cb.tm_grid[k] && cb.tm_grid[k] == grid) return k;
  return -1;
}

// TMA maps (slot `slot`) of cube cb's tile staging over the grid buffer `grid`
// ([L][K1][K2] float2).
void encode_cube_maps(Cube& cb, const float2* grid, int slot) {
  static EncodeTiledFn encode = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      encode = (EncodeTiledFn)fn;
  }
  {
    cb.tm_grid[slot] = nullptr;
    const int T = cb.tile, S = degrid_stage_stride(T);
    // the tile rows must lie in one t-slice of the view and the box must fit the grid
    const bool geom = (cb.N2c == 1 || cb.N1c == T) && T + kTaps - 1 <= 256 && S <= 256 && S <= cb.K2 &&
                      ((uintptr_t)grid % 16) == 0;
    if (!encode || !geom) return;
    cuuint64_t dims[4] = {(cuuint64_t)cb.K2, (cuuint64_t)cb.N2c, (cuuint64_t)cb.N1c, (cuuint64_t)cb.L};
    cuuint64_t strides[3] = {(cuuint64_t)cb.K2 * 8, (cuuint64_t)cb.N2c * cb.K2 * 8, (cuuint64_t)cb.K1 * cb.K2 * 8};
    cuuint32_t box_rows[4] = {(cuuint32_t)S, 1, (cuuint32_t)T, 1};
    cuuint32_t box_halo[4] = {(cuuint32_t)S, 1, (cuuint32_t)(kTaps - 1), 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r1 = encode(&cb.tm_rows[slot], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)grid, dims, strides,
                         box_rows, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    CUresult r2 = encode(&cb.tm_halo[slot], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4, (void*)grid, dims, strides,
                         box_halo, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r1 == CUDA_SUCCESS && r2 == CUDA_SUCCESS) cb.tm_grid[slot] = grid;
  }
}

// Deterministic pseudo-random values in [-1, 1) (an integer hash of the index), for the
// autotuner's trial inputs.
__global__ void k_fill_pattern(float* __restrict__ p, int64_t n, uint32_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 2654435761u ^ seed;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    p[i] = (float)(h >> 8) * (1.f / 8388608.f) - 1.f;
  }
}

void launch_fill_pattern(float* p, int64_t n, uint32_t seed, cudaStream_t st) {
  if (n <= 0) return;
  const unsigned g = (unsigned)std::min<int64_t>((n + 255) / 256, 4096);
  k_fill_pattern<<<g, 256, 0, st>>>(p, n, seed);
  note_launches(1);
}

cudaError_t set_wait_first(long long spins) {
  cudaError_t e = cudaMemcpyToSymbol(g_wait_first, &spins, sizeof(spins));
  if (e == cudaSuccess) e = set_gram_wait_first(spins);
  return e;
}

unsigned read_device_status(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_dev_status, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_dev_status, &z, sizeof(z));
  }
  return v | (read_gram_status(clear) << 8);
}

void launch_degrid(const Cube& cb, const float2* grid, float2* out, bool tiled, cudaStream_t st) {
  if (cb.dde_R >= 0) {
    launch_degrid_dde(cb, grid, out, st);
    return;
  }
  if (tiled) {
    dim3 grd(degrid_tiled_parts(cb), cb.L);
    const int ms = map_slot(cb, grid), k = ms < 0 ? 0 : ms;
    k_degrid_tiled<0><<<grd, 256, degrid_tiled_smem(cb), st>>>(grid, cb.d_uv, cb.d_tile_off, cb.d_vis_off,
                                                               vis_geom(cb), cb.tile, cb.ntile_r, cb.ntile_c, out,
                                                               nullptr, nullptr, nullptr, nullptr, cb.B, nullptr,
                                                               cb.tm_rows[k], cb.tm_halo[k], ms >= 0 ? 1 : 0);
  } else {
    dim3 grd(degrid_parts(cb), cb.L);
    k_degrid<<<grd, 256, 0, st>>>(grid, cb.d_uv, out, cb.d_vis_off, vis_geom(cb));
  }
  note_launches(1);
}

void launch_degrid_pdfb_tiled(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                              float2* u_prev, double* partials, cudaStream_t st) {
  dim3 grd(degrid_tiled_parts(cb), cb.L);
  const int ms = map_slot(cb, grid), k = ms < 0 ? 0 : ms;
  k_degrid_tiled<1><<<grd, 256, degrid_tiled_smem(cb), st>>>(grid, cb.d_uv, cb.d_tile_off, cb.d_vis_off,
                                                             vis_geom(cb), cb.tile, cb.ntile_r, cb.ntile_c, d_out, y,
                                                             v, u_prev, cb.d_blk, cb.B, partials, cb.tm_rows[k],
                                                             cb.tm_halo[k], ms >= 0 ? 1 : 0);
  note_launches(1);
}

void launch_degrid_pdfb(const Cube& cb, const float2* grid, const float2* y, const float2* v, float2* d_out,
                        float2* u_prev, double* partials, int nparts, cudaStream_t st) {
  dim3 grd(nparts, cb.L);
  k_degrid_pdfb<<<grd, 256, 0, st>>>(grid, cb.d_uv, y, v, d_out, u_prev, cb.d_blk, cb.d_vis_off, vis_geom(cb), cb.B,
                                     partials, nparts);
  note_launches(1);
}

void launch_l2ball_partials(const Cube& cb, const float2* z, const float2* y, float2* d, double* partials, int nparts,
                            cudaStream_t st) {
  dim3 grd(nparts, cb.L);
  k_l2ball_partials<<<grd, 256, 0, st>>>(z, y, d, cb.d_blk, cb.d_vis_off, cb.B, partials, nparts);
  note_launches(1);
}

void launch_block_finalize(const Cube& cb, const double* partials, int nparts, float* scale, double* out,
                           cudaStream_t st) {
  int n = cb.L * cb.B;
  k_block_finalize<<<n, 256, 0, st>>>(partials, nparts, cb.B, cb.L, cb.d_eps, scale, out);
  note_launches(1);
}

void launch_precond_duals(const Cube& cb, float2* d, float2* t, float* blk_scale, double* partials, cudaStream_t st) {
  const int np = degrid_parts(cb);
  dim3 grd(np, cb.L);
  for (int k = 0; k < cb.n_sub; ++k) {
    k_fb_step<<<grd, 256, 0, st>>>(d, t, cb.d_U, cb.d_gamma, blk_scale, cb.d_blk, cb.d_vis_off, cb.B, k == 0 ? 1 : 0,
                                   partials, np);
    launch_block_finalize(cb, partials, np, blk_scale, nullptr, st);
    note_launches(1);
  }
  k_fb_final<<<grd, 256, 0, st>>>(d, t, cb.d_U, blk_scale, cb.d_blk, cb.d_vis_off, cb.B);
  note_launches(1);
}

void launch_vis_scale(float2* v, const float* f, int64_t n, bool divide, cudaStream_t st) {
  if (n > 0) k_vis_scale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(v, f, n, divide ? 1 : 0);
  note_launches(1);
}

void launch_l2ball_scale(const Cube& cb, const float2* d, const float* scale, float2* v, cudaStream_t st) {
  dim3 grd(degrid_parts(cb), cb.L);
  k_l2ball_scale<<<grd, 256, 0, st>>>(d, scale, cb.d_blk, cb.d_vis_off, cb.B, v);
  note_launches(1);
}

void launch_grid(const Cube& cb, const float2* vals, const float* blk_scale, float2* v_write, float2* grid,
                 cudaStream_t st) {
  if (cb.dde_R >= 0) {
    launch_grid_dde(cb, vals, blk_scale, v_write, grid, st);
    return;
  }
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_grid<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024); attr = true; }
  dim3 grd(cb.ntile_r * cb.ntile_c, cb.L);
  size_t sm = 2 * (size_t)cb.tile * grid_row_stride(cb.tile) * sizeof(int);
  k_grid<0><<<grd, kGridThreads, sm, st>>>(vals, blk_scale, v_write, cb.d_uv, cb.d_blk, cb.d_tile_off, cb.d_vis_off, grid,
                                  cb.d_ncmax, vis_geom(cb), cb.tile, cb.ntile_r, cb.ntile_c, cb.B);
  note_launches(1);
}

void launch_grid_count(const Cube& cb, cudaStream_t st) {
  static bool attr = false;
  if (!attr) { cudaFuncSetAttribute(k_grid<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024); attr = true; }
  dim3 grd(cb.ntile_r * cb.ntile_c, cb.L);
  size_t sm = 2 * (size_t)cb.tile * grid_row_stride(cb.tile) * sizeof(int);
  k_grid<1><<<grd, kGridThreads, sm, st>>>(nullptr, nullptr, nullptr, cb.d_uv, cb.d_blk, cb.d_tile_off, cb.d_vis_off, nullptr,
                                  cb.d_ncmax, vis_geom(cb), cb.tile, cb.ntile_r, cb.ntile_c, cb.B);
  note_launches(1);
}

// ---------------------------------------------------- visibility reordering
__global__ void k_vis_gather(const int64_t* __restrict__ perm, int64_t n, const float2* __restrict__ in,
                             float2* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = in[perm[i]];
}

__global__ void k_vis_scatter(const int64_t* __restrict__ perm, int64_t n, const float2* __restrict__ in,
                              float2* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[perm[i]] = in[i];
}

void launch_vis_gather(const int64_t* perm, int64_t n, const float2* in, float2* out, cudaStream_t st) {
  if (n > 0) k_vis_gather<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(perm, n, in, out);
  note_launches(1);
}

void launch_vis_scatter(const int64_t* perm, int64_t n, const float2* in, float2* out, cudaStream_t st) {
  if (n > 0) k_vis_scatter<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(perm, n, in, out);
  note_launches(1);
}

void launch_measure(fhs_ctx* ctx, const Cube& cb, const float* x, float2* y, cudaStream_t st) {
  launch_fft_forward(ctx, cb, x, ctx->s.grid, st);
  launch_degrid(cb, ctx->s.grid, y, ctx->path == FHS_PATH_FAST && cb.degrid_tiled, st);
}

// host-side replica of kb_weights' first-tap rule (exact same float operations)
int host_first_tap(float om, int K) {
  TapConst t = tap_const(K, K);
  volatile float p = om * t.hi_r;
  volatile float q = p - 3.5f;
  return (int)floorf(q) + 1;
}

}  // namespace fhs

#include "dde.cuh"
