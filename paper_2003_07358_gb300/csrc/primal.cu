// Primal update of Algorithm 2 on GB300:
//   X+ = max(0, Re(X - tau A))  (Table 2, last row),  Xcheck = 2 X+ - X,
// with FP64 partial sums of ||X+ - X||^2 and ||X||^2 for the relative
// variation xi; float4 streaming, fixed grid, fixed-order reductions.
#include <cuda_runtime.h>

#include "fhs_internal.h"

namespace fhs {

constexpr int kPrimalCTAs = 1216;   // 152 SMs x 8

template <int NT>
__device__ __forceinline__ void cta_sum2(double a, double b, double* out) {
  __shared__ double s[2][NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s[0][wid] = a; s[1][wid] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int w = 0; w < NT / 32; ++w) { x += s[0][w]; y += s[1][w]; }
    out[0] = x;
    out[1] = y;
  }
}

// Compensated (Kahan) FP32 running sum; the FP64 pipe of the SM is kept for the
// final per-thread totals only.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

__global__ void __launch_bounds__(256) k_primal(float4* __restrict__ X, float4* __restrict__ Xc,
                                                const float4* __restrict__ A, float tau, int64_t n4,
                                                double* __restrict__ partials) {
  KahanF dx2, x2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
    float4 x = X[i], a = A[i];
    float4 xn;
    xn.x = fmaxf(0.f, fmaf(-tau, a.x, x.x));
    xn.y = fmaxf(0.f, fmaf(-tau, a.y, x.y));
    xn.z = fmaxf(0.f, fmaf(-tau, a.z, x.z));
    xn.w = fmaxf(0.f, fmaf(-tau, a.w, x.w));
    float4 xc;
    xc.x = 2.f * xn.x - x.x;
    xc.y = 2.f * xn.y - x.y;
    xc.z = 2.f * xn.z - x.z;
    xc.w = 2.f * xn.w - x.w;
    X[i] = xn;
    Xc[i] = xc;
    const float d0 = xn.x - x.x, d1 = xn.y - x.y, d2 = xn.z - x.z, d3 = xn.w - x.w;
    dx2.add(fmaf(d0, d0, fmaf(d1, d1, fmaf(d2, d2, d3 * d3))));
    x2.add(fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, x.w * x.w))));
  }
  cta_sum2<256>((double)dx2.s - (double)dx2.c, (double)x2.s - (double)x2.c, partials + 2 * blockIdx.x);
}

int primal_parts(const Cube&) { return kPrimalCTAs; }

void launch_primal(const Cube& cb, float* X, float* Xc, const float* A, double* partials, int nparts,
                   cudaStream_t st) {
  int64_t n = (int64_t)cb.L * cb.n1 * cb.n2;
  k_primal<<<nparts, 256, 0, st>>>((float4*)X, (float4*)Xc, (const float4*)A, (float)cb.tau, n / 4, partials);
  note_launches(1);
}

// Per-channel sums of squares: partials[l][p] over nparts CTAs per channel.
__global__ void __launch_bounds__(256) k_sumsq(const float* __restrict__ a, int64_t n, double* __restrict__ partials,
                                               int nparts) {
  const int l = blockIdx.y;
  const float* al = a + (size_t)l * n;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double v = al[i];
    s += v * v;
  }
  cta_sum2<256>(s, 0.0, partials + 2 * ((size_t)l * nparts + blockIdx.x));
}

void launch_sumsq(const float* a, int64_t n_per_ch, int L, double* partials, int nparts, cudaStream_t st) {
  dim3 g(nparts, L);
  k_sumsq<<<g, 256, 0, st>>>(a, n_per_ch, partials, nparts);
  note_launches(1);
}

__global__ void k_scale_ch(float* __restrict__ x, int64_t n, const double* __restrict__ inv) {
  const int l = blockIdx.y;
  float s = (float)inv[l];
  float* xl = x + (size_t)l * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xl[i] *= s;
}

void launch_scale_by_channel(float* x, int64_t n_per_ch, int L, const double* inv, cudaStream_t st) {
  dim3 g(64, L);
  k_scale_ch<<<g, 256, 0, st>>>(x, n_per_ch, inv);
  note_launches(1);
}

}  // namespace fhs
