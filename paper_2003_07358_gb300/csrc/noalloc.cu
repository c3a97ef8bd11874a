// Allocation-free variant of the l2-ball data-dual projection.
//
// Who needs it: callers that are not allowed to call cudaMalloc.  Examples: a
// host application that reserves all device memory up front in its own pool
// and hands plug-ins only pre-allocated buffers; a latency-critical loop where
// an allocation (and the implicit synchronisation it may bring) is not
// acceptable; a device whose memory is already fully committed.  Such a
// caller cannot create an fhs_ctx (fhs_create allocates tables and scratch),
// so this entry point takes plain arrays and keeps its only scratch -- the
// per-CTA partial sums of the block norms -- in a fixed-size array among the
// library's device globals.  Every GPU that loads the library holds that array
// (about 156 KB) until the process exits.
//
// Contract (see also include/fhs.h):
//  * no cudaMalloc, cudaFree or allocating library routine is called;
//  * at most kNoAllocMaxSeg segments per call; larger requests are rejected;
//  * the scratch array is shared by every call on a device and keeps the last
//    call's contents; each slot a call reads is first written by that same
//    call, so nothing has to be cleared between calls;
//  * calls whose kernels overlap on the GPU (e.g. on unordered streams) race
//    on the scratch array: the caller must serialise them;
//  * the first call on each device looks up the device address of the scratch
//    array with cudaGetSymbolAddress (the device must be current); make that
//    first call before any stream capture begins.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "fhs_internal.h"

namespace fhs {

constexpr int kNoAllocMaxSeg = 64;     // segments (data blocks) per call
constexpr int kNoAllocParts = 304;     // partial sums per segment (2 CTAs per SM)
constexpr int kNoAllocMaxDevices = 64;

// [seg][part] partial sums, then per segment {scale, ||z - y||}
static __device__ __align__(256) double g_l2_scratch[kNoAllocMaxSeg * kNoAllocParts + 2 * kNoAllocMaxSeg];

// Partial sums of ||z - y||^2 over [beg, end): one slot per CTA, CTAs without
// elements write 0, so every slot of the segment is written.
__global__ void __launch_bounds__(256) k_na_partials(const float2* __restrict__ z, const float2* __restrict__ y,
                                                     double* __restrict__ scratch, int64_t beg, int64_t end, int seg) {
  double s = 0.0;
  for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = z[i], b = y[i];
    double dx = (double)a.x - b.x, dy = (double)a.y - b.y;
    s += dx * dx + dy * dy;
  }
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    scratch[seg * kNoAllocParts + blockIdx.x] = t;
  }
}

// Fixed-order sum of a segment's partials; scale = max(0, 1 - eps / ||z - y||).
__global__ void k_na_segment_total(double* __restrict__ scratch, int seg, double eps) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int p = 0; p < kNoAllocParts; ++p) t += scratch[seg * kNoAllocParts + p];
  double dn = sqrt(t);
  double* fin = scratch + kNoAllocMaxSeg * kNoAllocParts;
  fin[2 * seg] = dn > eps ? 1.0 - eps / dn : 0.0;
  fin[2 * seg + 1] = dn;
}

// v = (z - y) * scale over the segment.
__global__ void k_na_scale(const float2* __restrict__ z, const float2* __restrict__ y, float2* __restrict__ v,
                           const double* __restrict__ scratch, int64_t beg, int64_t end, int seg) {
  const double* fin = scratch + kNoAllocMaxSeg * kNoAllocParts;
  float s = (float)fin[2 * seg];
  for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = z[i], b = y[i];
    v[i] = make_float2((a.x - b.x) * s, (a.y - b.y) * s);
  }
}

namespace {
std::mutex g_na_mu;
double* g_na_ptr[kNoAllocMaxDevices] = {nullptr};
thread_local std::string g_na_err;
}  // namespace

}  // namespace fhs

using namespace fhs;

extern "C" const char* fhs_noalloc_last_error(void) { return g_na_err.c_str(); }

extern "C" fhs_status fhs_proj_l2ball_noalloc(const float* z, const float* y, const int64_t* seg_off, int32_t nseg,
                                              const double* eps, float* v_out, double* dnorm_out, void* stream) {
  g_na_err.clear();
  if (!z || !y || !seg_off || !eps || !v_out) {
    g_na_err = "NULL argument";
    return FHS_ERR_INVALID_ARG;
  }
  if (nseg < 1 || nseg > kNoAllocMaxSeg) {
    g_na_err = "nseg must be in [1, " + std::to_string(kNoAllocMaxSeg) + "]: the static scratch holds " +
               std::to_string(kNoAllocMaxSeg) + " segments";
    return FHS_ERR_INVALID_ARG;
  }
  if (seg_off[0] < 0) {
    g_na_err = "segment offsets must start at >= 0";
    return FHS_ERR_INVALID_ARG;
  }
  for (int s = 0; s < nseg; ++s) {
    if (seg_off[s + 1] < seg_off[s] || !std::isfinite(eps[s]) || eps[s] < 0.0) {
      g_na_err = "segment offsets must be non-decreasing and radii finite and >= 0";
      return FHS_ERR_INVALID_ARG;
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    g_na_err = "no usable current CUDA device";
    return FHS_ERR_CUDA;
  }
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      // one-time set-up for this device: device address of the scratch array
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_l2_scratch);
      if (e != cudaSuccess) {
        g_na_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return FHS_ERR_CUDA;
      }
      g_na_ptr[dev] = (double*)p;
    }
    scratch = g_na_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float2* z2 = (const float2*)z;
  const float2* y2 = (const float2*)y;
  float2* v2 = (float2*)v_out;
  for (int s = 0; s < nseg; ++s) {
    k_na_partials<<<kNoAllocParts, 256, 0, st>>>(z2, y2, scratch, seg_off[s], seg_off[s + 1], s);
    k_na_segment_total<<<1, 32, 0, st>>>(scratch, s, eps[s]);
    int64_t n = seg_off[s + 1] - seg_off[s];
    unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * 152, (n + 255) / 256));
    k_na_scale<<<blocks, 256, 0, st>>>(z2, y2, v2, scratch, seg_off[s], seg_off[s + 1], s);
    note_launches(3);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    g_na_err = std::string("kernel launch: ") + cudaGetErrorString(e);
    return FHS_ERR_CUDA;
  }
  if (dnorm_out) {
    double fin[2 * kNoAllocMaxSeg];
    e = cudaMemcpyAsync(fin, scratch + kNoAllocMaxSeg * kNoAllocParts, 2 * (size_t)nseg * sizeof(double),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      g_na_err = std::string("reading the norms: ") + cudaGetErrorString(e);
      return FHS_ERR_CUDA;
    }
    for (int s = 0; s < nseg; ++s) {
      dnorm_out[s] = fin[2 * s + 1];
      if (!std::isfinite(dnorm_out[s])) {
        g_na_err = "non-finite block norm";
        return FHS_ERR_NONFINITE;
      }
    }
  }
  return FHS_OK;
}
