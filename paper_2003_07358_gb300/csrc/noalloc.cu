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
//    array with cudaGetSymbolAddress (the device must be current) and keeps it
//    for the life of the process; make that first call before any stream
//    capture begins, and do not reset the device (cudaDeviceReset) after it;
//  * a segment whose norm is NaN or Inf gets v = NaN (never a silent zero); the
//    status reports FHS_ERR_NONFINITE only when the norms are requested, since
//    only then does the call synchronise;
//  * with dnorm_out != NULL the call synchronises the stream, which is not
//    allowed while the stream is being captured: pass NULL there.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "fhs_internal.h"

namespace fhs {

constexpr int kNoAllocMaxSeg = 64;     // segments (data blocks) per call
constexpr int kNoAllocParts = 304;     // most partial sums per segment (the scratch row length)
constexpr int kNoAllocMaxDevices = 64;

// [seg][part] partial sums, then per segment {scale, ||z - y||}
static __device__ __align__(256) double g_l2_scratch[kNoAllocMaxSeg * kNoAllocParts + 2 * kNoAllocMaxSeg];

// Segment table passed by value (kernel parameter space, no device allocation).
struct NaSegs {
  int64_t off[kNoAllocMaxSeg + 1];
  double eps[kNoAllocMaxSeg];
};

// Partial sums of ||z - y||^2 of segment blockIdx.y: one slot per CTA of the row,
// CTAs without elements write 0, so every slot the total reads is written by this call.
__global__ void __launch_bounds__(256) k_na_partials(const float2* __restrict__ z, const float2* __restrict__ y,
                                                     double* __restrict__ scratch, const NaSegs segs) {
  const int seg = blockIdx.y;
  const int64_t beg = segs.off[seg], end = segs.off[seg + 1];
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

// One thread per segment: fixed-order sum of its `nparts` partials and the scale
// 1 - eps / ||z - y|| (0 inside the ball, the zero-norm case included).  A non-finite
// norm gives a NaN scale, so a NaN or Inf in z or y shows up as NaN in v instead of
// a silent zero.
__global__ void k_na_segment_total(double* __restrict__ scratch, int nseg, int nparts, const NaSegs segs) {
  const int seg = blockIdx.x * blockDim.x + threadIdx.x;
  if (seg >= nseg) return;
  double t = 0.0;
  for (int p = 0; p < nparts; ++p) t += scratch[seg * kNoAllocParts + p];
  const double dn = sqrt(t), eps = segs.eps[seg];
  double* fin = scratch + kNoAllocMaxSeg * kNoAllocParts;
  fin[2 * seg] = !isfinite(dn) ? nan("") : (dn > eps ? 1.0 - eps / dn : 0.0);
  fin[2 * seg + 1] = dn;
}

// v = (z - y) * scale over segment blockIdx.y.
__global__ void k_na_scale(const float2* __restrict__ z, const float2* __restrict__ y, float2* __restrict__ v,
                           const double* __restrict__ scratch, const NaSegs segs) {
  const int seg = blockIdx.y;
  const int64_t beg = segs.off[seg], end = segs.off[seg + 1];
  const double* fin = scratch + kNoAllocMaxSeg * kNoAllocParts;
  const float s = (float)fin[2 * seg];
  for (int64_t i = beg + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < end;
       i += (int64_t)gridDim.x * blockDim.x) {
    float2 a = z[i], b = y[i];
    v[i] = make_float2((a.x - b.x) * s, (a.y - b.y) * s);
  }
}

namespace {
std::mutex g_na_mu;
double* g_na_ptr[kNoAllocMaxDevices] = {nullptr};   // device address of g_l2_scratch per device
int g_na_parts[kNoAllocMaxDevices] = {0};           // partials per segment: 2 per SM, at most kNoAllocParts
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
  int parts = 0;
  {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
      // one-time set-up for this device: device address of the scratch array and
      // the number of partial sums per segment (two CTAs per SM)
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_l2_scratch);
      if (e != cudaSuccess) {
        g_na_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
        return FHS_ERR_CUDA;
      }
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess || sms < 1) {
        g_na_err = std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e);
        return FHS_ERR_CUDA;
      }
      g_na_parts[dev] = std::min(kNoAllocParts, 2 * sms);
      g_na_ptr[dev] = (double*)p;
    }
    scratch = g_na_ptr[dev];
    parts = g_na_parts[dev];
  }
  NaSegs segs;
  int64_t longest = 0;
  for (int s = 0; s <= nseg; ++s) segs.off[s] = seg_off[s];
  for (int s = 0; s < nseg; ++s) {
    segs.eps[s] = eps[s];
    longest = std::max<int64_t>(longest, seg_off[s + 1] - seg_off[s]);
  }
  cudaStream_t st = (cudaStream_t)stream;
  const float2* z2 = (const float2*)z;
  const float2* y2 = (const float2*)y;
  float2* v2 = (float2*)v_out;
  // three launches per call whatever the segment count: partials (segment = blockIdx.y),
  // one thread per segment for the totals, then the scaling
  k_na_partials<<<dim3(parts, nseg), 256, 0, st>>>(z2, y2, scratch, segs);
  k_na_segment_total<<<1, kNoAllocMaxSeg, 0, st>>>(scratch, nseg, parts, segs);
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(2 * parts, (longest + 255) / 256));
  k_na_scale<<<dim3(blocks, nseg), 256, 0, st>>>(z2, y2, v2, scratch, segs);
  note_launches(3);
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
