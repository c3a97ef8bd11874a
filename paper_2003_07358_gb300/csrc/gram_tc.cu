// Facet Gram matrices Z_q^T Z_q of the nuclear-norm duals on the 5th-generation tensor
// cores (tcgen05.mma, accumulator in tensor memory), error-free.
//
// The weighted nuclear prox (Algorithm 2 P update, Table 2 row 2) needs the L x L Gram
// of the facet matrix Z_q = P_q + D_q S~_q Xcheck (N~_q pixels x L channels), whose cost
// O(N~_q L^2) is the facet cores' SVD cost of Section 3.3.  A Gram from FP32 products
// accumulated in FP32 (or 3xTF32) has errors of order 2^-24 lambda_max, which the small
// singular values cannot afford; this kernel makes the contraction exact instead:
//
//  * per chunk of 1024 pixels and per channel a, z is scaled by 2^-(e_a + 1) with
//    2^e_a > max |z| (exact), and the scaled value r (|r| < 1/2) is cut into four
//    integer slices i_1..i_4, |i_k| <= 64:  r = sum_k i_k 128^-k + O(128^-4 / 2);
//  * the slices are exact bf16 values; one tcgen05.mma chain (M = N = 128, K = 16,
//    bf16 inputs, FP32 accumulation in TMEM) forms every slice-pair Gram
//    C[(k, a)][(m, b)] = sum_p i_ak(p) i_bm(p) of the chunk: integers below 2^22, exact
//    in FP32 whatever the accumulation order;
//  * the epilogue reads the accumulator (tcgen05.ld) and forms
//    G_ab = 2^(e_a + e_b + 2) sum_{k,m} 128^-(k+m) C[(k, a)][(m, b)] in exact 64-bit
//    fixed point (pairs with k + m <= 4), converted to FP64 once per entry.
//
// The only error is the 28-bit representation of z relative to its chunk-column
// maximum (~2^-29), far below the FP32 rounding of z itself.  Operand rows: 4 slices x
// 32 channels (L <= 32), or 2 half-chunks of 512 pixels x 4 slices x 16 channels
// (L <= 16; the two diagonal 64 x 64 blocks of C are used).
//
// Layout of an operand stage in shared memory (K-major, no swizzle, bf16): 4 MMA
// K-steps of 16; within a step, core matrices of 8 rows x 16 bytes, adjacent in K at
// 128 B (leading byte offset) and in rows at 256 B (stride byte offset).  A = B (the
// product is A A^T).  Every wait on the MMA's mbarrier is bounded: on timeout the
// kernel sets a status bit, waits (bounded) once more, frees its tensor memory and
// returns.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fhs_internal.h"

namespace fhs {

__device__ unsigned int g_gram_status = 0;
__device__ long long g_gram_wait_first = 0;   // first wait's length (0: kGramSpinLimit)
constexpr unsigned kGramTimeout = 1u;
constexpr long long kGramSpinLimit = 1ll << 24;

constexpr int kTcChunk = 1024;           // pixels per chunk (one FP64 partial, as k_gram)
constexpr int kTcStageK = 64;            // pixels (K) per operand stage: 4 MMA K-steps
constexpr int kTcRows = 128;             // M = N
constexpr int kTcStageBytes = kTcRows * kTcStageK * 2;   // 16 KB
constexpr int kTcThreads = 256;       // 8 warps; warps w and w + 4 share TMEM lanes

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start >> 4, leading byte offset >> 4 at bit
// 16, stride byte offset >> 4 at bit 32, descriptor version 1 at bit 46, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(unsigned saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::f16: D F32 (bit 4), A and B BF16 (bits 7, 10), both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcRows >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

__device__ __forceinline__ bool tc_mbar_wait(unsigned bar, unsigned parity, bool first = true) {
  const long long lim = !first ? kGramSpinLimit
                        : g_gram_wait_first > 0 ? g_gram_wait_first
                        : g_gram_wait_first < 0 ? 0 : kGramSpinLimit;
  for (long long it = 0; it < lim; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Slices of z * scale (|z * scale| < 1/2) as bf16 bit patterns: i_k, k = 1..4.
__device__ __forceinline__ void tc_slices(float z, float scale, unsigned short* s) {
  float r = z * scale;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float t = r * 128.f;                                       // exact
    const float i = __fsub_rn(__fadd_rn(t, 12582912.f), 12582912.f); // rint(t), |t| <= 64
    r = __fsub_rn(t, i);                                             // exact
    s[k] = (unsigned short)(__float_as_uint(i) >> 16);               // small integer: exact bf16
  }
}

// Paired FP32 arithmetic (add / sub / mul .rn.f32x2 of sm_100-family parts): the same
// IEEE round-to-nearest operation on both halves, two values per instruction.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// tc_slices of two values at once: s[k] holds slice k of z0 (low 16 bits) and of z1
// (high 16 bits) as bf16 bit patterns, the pair order of the operand rows.
__device__ __forceinline__ void tc_slices2(float z0, float z1, float scale, uint32_t* s) {
  const uint64_t c128 = f2_pack(128.f, 128.f), magic = f2_pack(12582912.f, 12582912.f);
  uint64_t r = f2_mul(f2_pack(z0, z1), f2_pack(scale, scale));
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint64_t t = f2_mul(r, c128);                       // exact
    const uint64_t i = f2_sub(f2_add(t, magic), magic);       // rint(t), |t| <= 64
    r = f2_sub(t, i);                                         // exact
    float i0, i1;
    f2_unpack(i, i0, i1);
    s[k] = __byte_perm(__float_as_uint(i0), __float_as_uint(i1), 0x7632);
  }
}

// Value of facet pixel (rr, cc) (linear index p < Nq), channel l: D_q Xcheck + P_q.
__device__ __forceinline__ float tc_z(const float* __restrict__ xc, const float* __restrict__ P, const NucFacet& f,
                                      float d, size_t xo, size_t N, int Nq, int use_P, int p, int l) {
  float v = d * xc[(size_t)l * N + xo];
  if (use_P) v += P[f.p_off + (size_t)l * Nq + p];
  return v;
}

// LP = 16 (two half-chunks side by side) or 32 (one chunk).  Grid (chunks, facets).
// Pass 1 reads the chunk for the per-(half-chunk, channel) maxima; pass 2 reads it again
// (from L2) and cuts the operand stages, double-buffered against the MMAs.  Shared
// memory: two operand stages (32 KB), reused by the epilogue's reduction.
template <int LP>
__global__ void __launch_bounds__(kTcThreads, 2) k_gram_tc(const float* __restrict__ xc, const float* __restrict__ P,
                                                        const NucFacet* __restrict__ facets,
                                                        const float* __restrict__ win, int n1, int n2, int L,
                                                        int use_P, double* __restrict__ part, int nchunk_max) {
  constexpr int NH = 32 / LP;                  // half-chunks per MMA row block (2 or 1)
  constexpr int HP = kTcChunk / NH;            // pixels per half-chunk
  constexpr int RH = 4 * LP;                   // operand rows per half-chunk (64 or 128)
  constexpr int NSTAGE = HP / kTcStageK;       // operand stages per chunk (8 or 16)
  constexpr int NTASK = NH * LP * (kTcStageK / 8);   // (half, channel, 8 pixels) tasks per stage
  // LP = 16: the chunk's values are loaded once (coalesced) into a shared stash, then
  // reduced and sliced from there; LP = 32: read twice from global memory (the second
  // pass hits L2), which keeps the shared memory at two operand stages
  constexpr bool STASH = LP == 16;
  static_assert(NTASK == kTcThreads, "one slicing task per thread and stage");
  static_assert((size_t)NH * 4 * LP * LP * sizeof(double) <= 2 * (size_t)kTcStageBytes,
                "the epilogue reduction reuses the operand buffers");
  extern __shared__ __align__(128) unsigned char tc_smem[];
  unsigned char* opnd = tc_smem;                                                 // 2 stages
  float* zs = reinterpret_cast<float*>(tc_smem + 2 * kTcStageBytes);             // STASH: [LP][kTcChunk]
  double* red = reinterpret_cast<double*>(tc_smem);                              // [NH][4][LP][LP]
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ __align__(8) uint64_t mbar_drain;  // completes when every MMA issued so far has
  __shared__ uint32_t tmem_base;
  __shared__ int s_max[NH][LP];                // per (half-chunk, channel) max |z| (float bits)
  __shared__ float s_scale[NH][LP];
  __shared__ double s_pow[NH][LP];             // 2^(e + 1)
  __shared__ __align__(16) int2 s_px[kTcChunk];  // per chunk pixel: window weight d (bits), image offset

  const int q = blockIdx.y, chunk = blockIdx.x;
  const NucFacet f = facets[q];
  const int w = f.c1 - f.c0, Nq = (f.r1 - f.r0) * w;
  const int p0 = chunk * kTcChunk;
  if (p0 >= Nq) return;                        // whole CTA: before any allocation
  const size_t N = (size_t)n1 * n2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  // ---- tensor memory (128 columns: the 128 x 128 FP32 accumulator) and mbarriers
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(128u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar[1])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&mbar_drain)));
    asm volatile("fence.mbarrier_init.release.cluster;\n");
  }
  for (int i = tid; i < NH * LP; i += kTcThreads) (&s_max[0][0])[i] = 0;
  __syncthreads();

  if constexpr (STASH) {
    // ---- pass 1: thread = pixel, all channels (coalesced along the facet row) into
    // the stash; then thread (half, channel, 8-pixel segment) takes the maximum of the
    // 64 values it slices later, 8 lanes per (half, channel)
#pragma unroll
    for (int j = 0; j < kTcChunk / kTcThreads; ++j) {
      const int qq = tid + j * kTcThreads, p = p0 + qq;
      if (p < Nq) {
        const int rr = p / w, cc = p - rr * w;
        const float d = win[f.wy_off + rr] * win[f.wx_off + cc];
        const size_t xo = (size_t)(f.r0 + rr) * n2 + (f.c0 + cc);
#pragma unroll
        for (int l = 0; l < LP; ++l) zs[l * kTcChunk + qq] = l < L ? tc_z(xc, P, f, d, xo, N, Nq, use_P, p, l) : 0.f;
      } else {
#pragma unroll
        for (int l = 0; l < LP; ++l) zs[l * kTcChunk + qq] = 0.f;
      }
    }
    __syncthreads();
    const int sg = tid % (kTcStageK / 8), shl = tid / (kTcStageK / 8);
    const int stl = shl % LP, sth = shl / LP;
    float m = 0.f;
#pragma unroll
    for (int st2 = 0; st2 < NSTAGE; ++st2) {
      const float4* z4 = reinterpret_cast<const float4*>(zs + stl * kTcChunk + sth * HP + st2 * kTcStageK + sg * 8);
      const float4 a = z4[0], b = z4[1];
      m = fmaxf(m, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
      m = fmaxf(m, fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w))));
    }
#pragma unroll
    for (int o = 1; o < kTcStageK / 8; o <<= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (sg == 0) s_max[sth][stl] = __float_as_int(m);
  } else {
  // ---- pass 1: thread = pixel (one division, one window weight), all channels
  // (coalesced along the facet row); maxima in registers, warp shuffles, one shared
  // atomic per warp and (half, channel)
  {
    float mx[NH][LP];
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
      for (int l = 0; l < LP; ++l) mx[h][l] = 0.f;
#pragma unroll
    for (int j = 0; j < kTcChunk / kTcThreads; ++j) {
      constexpr int JH = HP / kTcThreads;              // iterations per half-chunk
      const int h = j / JH;                            // compile-time after unrolling
      const int p = p0 + tid + j * kTcThreads;
      int2 px = make_int2(0, 0);
      if (p < Nq) {
        const int rr = p / w, cc = p - rr * w;
        const float d = win[f.wy_off + rr] * win[f.wx_off + cc];
        const int xo = (f.r0 + rr) * n2 + (f.c0 + cc);     // < 2^24 (n1, n2 <= 4096)
        px = make_int2(__float_as_int(d), xo);
#pragma unroll
        for (int l = 0; l < LP; ++l)
          if (l < L) mx[h][l] = fmaxf(mx[h][l], fabsf(tc_z(xc, P, f, d, (size_t)xo, N, Nq, use_P, p, l)));
      }
      s_px[tid + j * kTcThreads] = px;
    }
#pragma unroll
    for (int h = 0; h < NH; ++h)
#pragma unroll
      for (int l = 0; l < LP; ++l) {
        float m = mx[h][l];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0 && l < L) atomicMax(&s_max[h][l], __float_as_int(m));
      }
  }
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  const uint32_t tmem = tmem_base;
  for (int i = tid; i < NH * LP; i += kTcThreads) {
    const float m = __int_as_float((&s_max[0][0])[i]);
    int e = 0;
    if (m > 0.f) frexpf(m, &e);                // m = f 2^e, f in [1/2, 1): m < 2^e
    (&s_scale[0][0])[i] = m > 0.f ? ldexpf(1.f, -(e + 1)) : 1.f;
    (&s_pow[0][0])[i] = m > 0.f ? ldexp(1.0, e + 1) : 1.0;
  }
  __syncthreads();

  // ---- pass 2: operand stages (double-buffered) and the MMA chain.  Thread task:
  // (half h, channel l, segment of 8 consecutive pixels) -> 4 slice rows x 16 B
  const int seg = tid % (kTcStageK / 8), hl = tid / (kTcStageK / 8);
  const int tl = hl % LP, th = hl / LP;
  const int k0 = seg * 8;                      // K offset within a stage
  const bool chan = tl < L;
  const float sc = s_scale[th][tl];
  bool ok = true;
  unsigned phase[2] = {0u, 0u};
  // the 8 values of a stage (window weights and offsets from the pixel table); stage
  // s + 1's loads are issued before stage s is sliced
  const float* xcl = xc + (size_t)(chan ? tl : 0) * N;
  const float* Pl = use_P ? P + f.p_off + (size_t)(chan ? tl : 0) * Nq : P;
  auto load8 = [&](int s, float* zv) {
    const int q0 = th * HP + s * kTcStageK + k0;       // chunk-local pixel
    if constexpr (STASH) {
      const float4* z4 = reinterpret_cast<const float4*>(zs + tl * kTcChunk + q0);
      const float4 a = z4[0], b = z4[1];
      zv[0] = a.x; zv[1] = a.y; zv[2] = a.z; zv[3] = a.w;
      zv[4] = b.x; zv[5] = b.y; zv[6] = b.z; zv[7] = b.w;
      return;
    }
    const int4* t4 = reinterpret_cast<const int4*>(s_px + q0);
#pragma unroll
    for (int jj = 0; jj < 4; ++jj) {
      const int4 e = t4[jj];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int p = p0 + q0 + 2 * jj + u;
        float v = 0.f;
        if (chan && p < Nq) {
          v = __int_as_float(u ? e.z : e.x) * xcl[u ? e.w : e.y];
          if (use_P) v += Pl[p];
        }
        zv[2 * jj + u] = v;
      }
    }
  };
  float zn[8];
  load8(0, zn);
  for (int s = 0; s < NSTAGE; ++s) {
    const int buf = s & 1;
    unsigned char* ob = opnd + buf * kTcStageBytes;
    float zv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) zv[j] = zn[j];
    if (s + 1 < NSTAGE) load8(s + 1, zn);
    if (s >= 2) {   // the MMAs of stage s - 2 read this buffer
      if (!tc_mbar_wait(smem_u32(&mbar[buf]), phase[buf])) { ok = false; }
      phase[buf] ^= 1u;
    }
    if (__syncthreads_or(!ok)) { ok = false; break; }
    uint32_t sl[4][4];                          // [pixel pair][slice]
#pragma unroll
    for (int j = 0; j < 4; ++j) tc_slices2(zv[2 * j], zv[2 * j + 1], sc, sl[j]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int row = th * RH + k * LP + tl;
      const int off = (k0 / 16) * 4096 + ((k0 / 8) & 1) * 128 + (row / 8) * 256 + (row % 8) * 16;
      *reinterpret_cast<uint4*>(ob + off) = make_uint4(sl[0][k], sl[1][k], sl[2][k], sl[3][k]);
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (tid == 0) {
      const unsigned obase = smem_u32(ob);
#pragma unroll
      for (int ks = 0; ks < kTcStageK / 16; ++ks) {
        const uint64_t d = tc_smem_desc(obase + ks * 4096);
        const unsigned acc = (s > 0 || ks > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(d), "l"(d), "r"(kTcIdesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar[buf]))
                   : "memory");
    }
  }
  // the commits of the last two stages are still pending; the last covers every MMA
  if (ok) {
    const int last = (NSTAGE - 1) & 1;
    if (!tc_mbar_wait(smem_u32(&mbar[last ^ 1]), phase[last ^ 1])) ok = false;
    if (ok && !tc_mbar_wait(smem_u32(&mbar[last]), phase[last])) ok = false;
  }
  if (__syncthreads_or(!ok)) {
    // a wait gave up: flag it, give the MMAs a second bounded chance to land, then free
    // the tensor memory and leave (the partial of this chunk is not written)
    // (the threads may disagree on the pending phases of mbar[]: a fresh commit to the
    // drain barrier tracks every MMA issued so far, and its first phase is the one)
    if (tid == 0) {
      atomicOr(&g_gram_status, kGramTimeout);
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&mbar_drain))
                   : "memory");
    }
    tc_mbar_wait(smem_u32(&mbar_drain), 0u, false);
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128u));
    return;
  }
  asm volatile("tcgen05.fence::after_thread_sync;\n");

  // ---- epilogue: warp w reads TMEM lanes 32 (w % 4) + lane = row i of C, columns of
  // its half of the row's block (warps w and w + 4 split them); i = h RH + k LP + a.
  // The slice-pair sums C are exact integers (< 2^22); they are combined exactly in
  // 64-bit fixed point, T = sum_{k+m <= 4} C_km 2^(7 (4 - k - m)) (value T 2^-42; the
  // pairs with k + m >= 5 weigh below 2^-35 of the leading pair and are left out), and
  // converted to FP64 once per Gram entry (FP64 is slow on this part).
  long long T[LP];
  const int i = (warp & 3) * 32 + lane;
  const int h = i / RH, k = (i % RH) / LP, a = i % LP;
  const int half = warp >> 2;
#pragma unroll
  for (int b = 0; b < LP; ++b) T[b] = 0;
#pragma unroll
  for (int c16 = 0; c16 < RH / 32; ++c16) {
    const int cb = half * (RH / 2) + c16 * 16;     // column within this half-chunk's block
    uint32_t v[16];
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(h * RH + cb);
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int col = cb + t;                      // m LP + b
      const int m = col / LP, b = col % LP;
      const int sh = 7 * (4 - k - m);
      // exact integer of a float below 2^22 by one FP32 add (full rate)
      const int c = __float_as_int(__fadd_rn(__uint_as_float(v[t]), 12582912.f)) - 0x4B400000;
      if (sh >= 0) T[b] += (long long)c << sh;
    }
  }
  // integer sums: exact in any order; the first column half writes, the second adds
  long long* ired = reinterpret_cast<long long*>(red);
  long long* r = ired + (((size_t)h * 4 + k) * LP + a) * LP;
  if (half == 0) {
#pragma unroll
    for (int b = 0; b < LP; ++b) r[b] = T[b];
  }
  __syncthreads();
  if (half == 1) {
#pragma unroll
    for (int b = 0; b < LP; ++b) r[b] += T[b];
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(128u));
  // sum over slices k (exact), then per half-chunk the scales 2^(e_a + 1) 2^(e_b + 1) 2^-42
  double* out = part + ((size_t)q * nchunk_max + chunk) * L * L;
  for (int ab = tid; ab < L * L; ab += kTcThreads) {
    const int a2 = ab / L, b2 = ab % L;
    double g = 0.0;
    for (int hh = 0; hh < NH; ++hh) {
      long long gh = 0;
      for (int kk = 0; kk < 4; ++kk) gh += ired[(((size_t)hh * 4 + kk) * LP + a2) * LP + b2];
      g += (double)gh * (s_pow[hh][a2] * s_pow[hh][b2] * 0x1p-42);
    }
    out[ab] = g;
  }
}

static size_t gram_tc_smem(int LP) {
  return 2 * (size_t)kTcStageBytes + (LP == 16 ? (size_t)LP * kTcChunk * sizeof(float) : 0);
}

bool launch_gram_tc(const Cube& cb, const float* xcheck, const float* P, double* part, int nchunk_max,
                    cudaStream_t st) {
  if (cb.L > 32) return false;
  dim3 grd(nchunk_max, cb.Qy * cb.Qx);
  const int use_P = P != nullptr ? 1 : 0;
  if (cb.L <= 16) {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gram_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem(16));
      attr = true;
    }
    k_gram_tc<16><<<grd, kTcThreads, gram_tc_smem(16), st>>>(xcheck, P, cb.d_facets, cb.d_win, cb.n1, cb.n2, cb.L,
                                                             use_P, part, nchunk_max);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_gram_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram_tc_smem(32));
      attr = true;
    }
    k_gram_tc<32><<<grd, kTcThreads, gram_tc_smem(32), st>>>(xcheck, P, cb.d_facets, cb.d_win, cb.n1, cb.n2, cb.L,
                                                             use_P, part, nchunk_max);
  }
  note_launches(1);
  return true;
}

cudaError_t set_gram_wait_first(long long spins) {
  return cudaMemcpyToSymbol(g_gram_wait_first, &spins, sizeof(spins));
}

unsigned read_gram_status(bool clear) {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_gram_status, sizeof(v)) != cudaSuccess) return 0;
  if (clear && v) {
    const unsigned z = 0;
    cudaMemcpyToSymbol(g_gram_status, &z, sizeof(z));
  }
  return v;
}

}  // namespace fhs
